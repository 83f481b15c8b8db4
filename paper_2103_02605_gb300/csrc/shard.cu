// shard.cu -- fcirc_batched_partition: the split of a batch of independent
// f-circulant products over several ranks (one GPU each).
//
// A batch's instances share nothing, as the two halves of one product share
// nothing after a halving step (the structure argument in the proof of
// Theorem 1, Section 2), so ranks need no exchange: each takes a subset and
// runs fcirc_matvec_batched on it.  The subsets come from the longest-
// processing-time rule on the cost of Algorithm 1 per instance, n log2 n,
// computed identically by every rank.  Host code only.
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/fcirc.h"
#include "common.hpp"

namespace fcirc {
namespace {

// The work of Algorithm 1 on an instance of size n: log2 n halving levels of
// n/2 butterflies for each of three trees, so proportional to n log2 n
// (taken as n below n = 2, and for sizes between powers of two by the
// ceiling of the logarithm).
double instance_cost(uint64_t n)
{
    int lg = 0;
    while (lg < 64 && ((uint64_t)1 << lg) < n) ++lg;
    return (double)n * (double)(lg > 1 ? lg : 1);
}

}  // namespace
}  // namespace fcirc

using namespace fcirc;

extern "C" int fcirc_batched_partition(const uint64_t *offsets, uint32_t count, uint32_t nranks, uint32_t rank,
                                       uint32_t *members, uint32_t *nmembers, double *loads)
{
    set_error("");
    if (!offsets || !nmembers || (count > 0 && !members))
        return fail(FCIRC_EINVAL, "fcirc_batched_partition: null pointer");
    if (nranks == 0 || nranks > 65536 || rank >= nranks)
        return fail(FCIRC_EINVAL, "fcirc_batched_partition: rank %u of %u ranks", rank, nranks);
    for (uint32_t i = 0; i < count; ++i)
        if (offsets[i + 1] < offsets[i])
            return fail(FCIRC_EINVAL, "fcirc_batched_partition: offsets decrease at instance %u", i);
    try {
        std::vector<uint32_t> order(count);
        std::vector<double> cost(count);
        for (uint32_t i = 0; i < count; ++i) {
            order[i] = i;
            cost[i] = instance_cost(offsets[i + 1] - offsets[i]);
        }
        // largest cost first; equal costs in index order (a total order, so
        // every rank sorts identically)
        std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
            return cost[a] != cost[b] ? cost[a] > cost[b] : a < b;
        });
        std::vector<double> load(nranks, 0.0);
        std::vector<uint32_t> owner(count);
        for (uint32_t k = 0; k < count; ++k) {
            uint32_t best = 0;
            for (uint32_t r = 1; r < nranks; ++r)
                if (load[r] < load[best]) best = r;
            owner[order[k]] = best;
            load[best] += cost[order[k]];
        }
        uint32_t m = 0;
        for (uint32_t i = 0; i < count; ++i)
            if (owner[i] == rank) members[m++] = i;
        *nmembers = m;
        if (loads)
            for (uint32_t r = 0; r < nranks; ++r) loads[r] = load[r];
    } catch (const std::bad_alloc &) {
        return fail(FCIRC_ENOMEM, "fcirc_batched_partition: host allocation of %u entries failed", count);
    }
    return FCIRC_OK;
}
