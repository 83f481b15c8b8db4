// Host build of the device arithmetic headers (modarith.cuh, gfp2.hpp,
// ssa.cuh) for tests/test_host_arith.py: reads one operation per line on
// stdin, writes its result.  The CUDA qualifiers are defined away; the one
// device intrinsic the headers use (__umul64hi) gets a 128-bit host version.
#include <stdint.h>
#include <cstdio>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
#define __ldg(p) (*(p))
#include "../../paper_2103_02605_gb300/csrc/modarith.cuh"
#include "../../paper_2103_02605_gb300/csrc/gfp2.hpp"
#include "../../paper_2103_02605_gb300/csrc/ssa.cuh"
#include "../../paper_2103_02605_gb300/csrc/ring.hpp"

using namespace fcirc;

template <int W>
static SsaE<W> rd()
{
    SsaE<W> e;
    for (int i = 0; i < W; ++i) scanf("%lx", &e.w[i]);
    scanf("%lx", &e.top);
    return e;
}
template <int W>
static void pr(const SsaE<W> &e)
{
    for (int i = 0; i < W; ++i) printf("%lx ", e.w[i]);
    printf("%lx\n", e.top);
}
template <int W>
static void ssa_op(const char *op)
{
    if (!strcmp(op, "add")) { auto a = rd<W>(), b = rd<W>(); pr<W>(cadd<W>(a, b)); }
    else if (!strcmp(op, "sub")) { auto a = rd<W>(), b = rd<W>(); pr<W>(csub<W>(a, b)); }
    else if (!strcmp(op, "neg")) { auto a = rd<W>(); pr<W>(cneg<W>(a)); }
    else if (!strcmp(op, "mul")) { auto a = rd<W>(), b = rd<W>(); pr<W>(cmul<W>(a, b)); }
    else { int e; scanf("%d", &e); auto a = rd<W>(); pr<W>(cmul<W>(SsaTw<W>{e}, a)); }
}

int main()
{
    char kind[8], op[8];
    while (scanf("%7s %7s", kind, op) == 2) {
        if (!strcmp(kind, "ssa1") || !strcmp(kind, "ssa2")) {
            if (kind[3] == '1') ssa_op<1>(op); else ssa_op<2>(op);
        } else if (!strcmp(kind, "gf")) {
            if (!strcmp(op, "red")) {
                unsigned long long x;
                scanf("%llx", &x);
                printf("%u\n", gf::red(x));
            } else {
                unsigned a, b, c, d;
                scanf("%u %u %u %u", &a, &b, &c, &d);
                const gf::E x{a, b}, y{c, d};
                gf::E r = !strcmp(op, "mul") ? gf::mul(x, y) : !strcmp(op, "add") ? gf::add(x, y)
                        : !strcmp(op, "sub") ? gf::sub(x, y) : gf::neg(x);
                printf("%u %u\n", r.re, r.im);
            }
        } else if (!strcmp(kind, "mod")) {
            // mod <op> p w x y z ...: 32-bit arithmetic mod p (p < 2^30; the
            // Barrett products take p < 2^31)
            unsigned p;
            scanf("%u", &p);
            const uint32_t p2 = 2 * p;
            if (!strcmp(op, "shoup")) {
                unsigned x, w;
                scanf("%u %u", &x, &w);
                printf("%u\n", shoup_mul(x, w, (uint32_t)(((uint64_t)w << 32) / p), p));
            } else if (!strcmp(op, "barrett")) {
                // the plan kernel's products and powers: ModP (ring.hpp)
                unsigned a, b;
                unsigned long long e;
                scanf("%u %u %llu", &a, &b, &e);
                const host::ModP M(p);
                printf("%u %u\n", M.mul(a, b), M.pow(a, e));
            } else if (!strcmp(op, "bquot")) {
                // Barrett quotients: floor(w 2^32 / p) and floor(w 2^64 / p)
                unsigned w;
                scanf("%u", &w);
                const host::ModP M(p);
                uint32_t hi, lo;
                M.quot64(w, hi, lo);
                printf("%u %u %u\n", M.quot32(w), hi, lo);
            } else if (!strcmp(op, "root")) {
                // a 2^k-th root by the Barrett path, and by the plain path
                unsigned f, Om;
                int k, v;
                scanf("%u %d %u %d", &f, &k, &Om, &v);
                uint32_t r1 = 0, r2 = 0;
                const bool o1 = host::nth_root_2k_om(f, k, host::ModP(p), Om, v, r1);
                const bool o2 = host::nth_root_2k_om(f, k, p, Om, v, r2);
                printf("%d %u %d %u\n", (int)o1, r1, (int)o2, r2);
            } else if (!strcmp(op, "redc")) {
                unsigned long long t;
                unsigned pinv;
                scanf("%llx %u", &t, &pinv);
                printf("%u\n", redc(t, p, pinv));
            } else if (!strcmp(op, "leaf")) {
                // two sibling leaves (parameters +s and -s), the row shifted by one place:
                // leaf2, swap, then level-L-1 recombination with bfly_rec / bfly_rec_shift
                unsigned a[4], y[4], s, si, pinv;
                for (int i = 0; i < 4; ++i) scanf("%u", &a[i]);
                for (int i = 0; i < 4; ++i) scanf("%u", &y[i]);
                scanf("%u %u %u", &s, &si, &pinv);
                const Tw ts{s, (uint32_t)(((uint64_t)s << 32) / p)};
                const Tw tsi{si, (uint32_t)(((uint64_t)si << 32) / p)};
                uint32_t A0 = a[0], A1 = a[1], B0 = a[2], B1 = a[3];
                leaf2(A0, A1, y[0], y[1], ts, p, p2, pinv);
                leaf2(B0, B1, y[2], y[3], tw_neg(ts, p), p, p2, pinv);
                uint32_t t;
                t = A0; A0 = A1; A1 = t;
                t = B0; B0 = B1; B1 = t;
                bfly_rec(A0, B0, tsi, p, p2);
                bfly_rec_shift(A1, B1, ts, p, p2);
                printf("%u %u %u %u\n", A0 % p, A1 % p, B0 % p, B1 % p);
            }
        }
        fflush(stdout);
    }
    return 0;
}
