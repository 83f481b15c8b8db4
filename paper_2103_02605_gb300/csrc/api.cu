// api.cu -- the C ABI (include/fcirc.h): argument checks, host/device
// staging, and the pass sequence of each entry point.
#include <stdio.h>
#include <string.h>

#include <cmath>

#include <chrono>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.hpp"
#include "kernels_batched.hpp"
#include "kernels_bigint.hpp"
#include "kernels_complex.hpp"
#include "kernels_mod.hpp"
#include "prof.hpp"
#include "gfp2.hpp"
#include "ring.hpp"

namespace fcirc {

const char *last_error_detail();

// ---------------------------------------------------------------------------
// host / device arguments

namespace {

struct Arg {
    const void *user;   // caller pointer
    size_t bytes;
    bool in, out;
    bool on_device = false;
    bool pinned = false;        // page-locked host memory
    void *d = nullptr;          // device pointer used by the kernels
};

int classify(Arg &a)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, a.user);
    a.pinned = false;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        a.on_device = false;
        return FCIRC_OK;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
        int dev = 0;
        FCIRC_CUDA_TRY(cudaGetDevice(&dev));
        if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
            return fail(FCIRC_EINVAL, "pointer %p lives on device %d, current device is %d", a.user,
                        attr.device, dev);
        a.on_device = true;
    } else {
        a.on_device = false;
        a.pinned = attr.type == cudaMemoryTypeHost;
    }
    return FCIRC_OK;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Stages host arguments through the scratch pool; `extra` bytes of compute
// scratch follow the staging area.  With page-locked host buffers only, the
// copies stay asynchronous on the stream (cudaMemcpyAsync semantics); any
// pageable host buffer makes end() wait for the stream.
struct Staging {
    std::vector<Arg *> args;
    cudaStream_t s;
    char *scratch = nullptr;
    bool any_host = false;
    bool any_pageable = false;

    int begin(cudaStream_t st, size_t extra)
    {
        s = st;
        size_t need = 0;
        for (Arg *a : args) {
            FCIRC_TRY(classify(*a));
            if (!a->on_device) {
                any_host = true;
                any_pageable = any_pageable || !a->pinned;
                need += align256(a->bytes);
            }
        }
        need += align256(extra);
        void *base = nullptr;
        if (need) FCIRC_TRY(scratch_acquire(s, need, &base));
        char *cur = static_cast<char *>(base);
        for (Arg *a : args) {
            if (a->on_device) {
                a->d = const_cast<void *>(a->user);
            } else {
                a->d = cur;
                cur += align256(a->bytes);
                if (a->in && a->bytes) {
                    ProfScope ps("copy_h2d", s);
                    FCIRC_CUDA_TRY(cudaMemcpyAsync(a->d, a->user, a->bytes, cudaMemcpyHostToDevice, s));
                }
            }
        }
        scratch = cur;
        return FCIRC_OK;
    }

    int end()
    {
        if (!any_host) return FCIRC_OK;
        for (Arg *a : args)
            if (!a->on_device && a->out && a->bytes) {
                ProfScope ps("copy_d2h", s);
                FCIRC_CUDA_TRY(cudaMemcpyAsync(const_cast<void *>(a->user), a->d, a->bytes,
                                               cudaMemcpyDeviceToHost, s));
            }
        if (any_pageable) FCIRC_CUDA_TRY(cudaStreamSynchronize(s));
        return FCIRC_OK;
    }
};

CrtConsts make_crt(uint32_t p1, uint32_t p2, uint32_t p3)
{
    using namespace host;
    CrtConsts C;
    C.p1 = p1;
    C.p2 = p2;
    C.p3 = p3;
    C.m2 = (uint32_t)((((uint64_t)1) << 32) / p2);
    C.m3 = (uint32_t)((((uint64_t)1) << 32) / p3);
    auto tw = [](uint32_t w, uint32_t p) {
        Tw t;
        t.w = w % p;
        t.wp = shoup_quot(t.w, p);
        return t;
    };
    C.inv12 = tw(invmod(p1 % p2, p2), p2);
    C.p1m3 = tw(p1 % p3, p3);
    C.inv123 = tw(invmod(mulmod(p1 % p3, p2 % p3, p3), p3), p3);
    C.p1p2 = (uint64_t)p1 * p2;
    return C;
}

TileJob tile_job(const Plan *pl, Src a, Src x, uint32_t *dst, int lazy)
{
    TileJob J;
    J.a = a;
    J.x = x;
    J.dst = dst;
    J.sig = pl->d_sig;
    J.rho = pl->d_rho;
    J.U = pl->pt->d_U;
    J.Ui = pl->pt->d_Ui;
    J.p = pl->p;
    J.pinv = pl->pt->pinv;
    J.store_lazy = lazy;
    return J;
}

// Pass dispatch: the register-staged kernels where their shapes apply, the
// generic shared-memory kernels otherwise.
int run_tile(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s)
{
    return fast_tile_ok(P.logT) ? launch_tile_fast(P, ntiles, njobs, s) : launch_tile(P, ntiles, njobs, s);
}

// One forward strided pass (pass index `pass` of the plans' shape) for
// `njobs` (source, destination, plan) jobs; the register-staged kernel runs
// `jobs_per_cta` of them in one CTA when its shape applies.
struct FwdDesc {
    Src src;
    uint32_t *dst;
    const Plan *pl;
    int vec_side;
    int half;
};

// The register-staged column pass parameters of forward pass `pass`; false
// when the pass's shape needs the generic strided kernels.
bool fwd_params(int pass, const FwdDesc *jd, int njobs, int jobs_per_cta, ColFwdParams &P)
{
    const Plan &sh = *jd[0].pl;
    const int l0 = sh.pass_l0[pass], l1 = sh.pass_l1[pass];
    if (!fast_col_ok(l1 - l0, sh.m - l1)) return false;
    P = ColFwdParams{};
    for (int k = 0; k < njobs; ++k)
        P.job[k] = ColFwdJob{jd[k].src, jd[k].dst, jd[k].pl->d_gtw + jd[k].pl->pass_goff[pass], jd[k].pl->p,
                             jd[k].vec_side, jd[k].half, jd[k].pl->d_gtwl + jd[k].pl->pass_loff[pass]};
    P.jobs_per_cta = jobs_per_cta;
    P.N = (uint32_t)sh.n;
    P.logn = sh.m;
    P.l0 = l0;
    P.l1 = l1;
    for (int st = 0; st < 3; ++st) P.stage_off[st] = sh.stage_off[pass][st];
    return true;
}

// ilv: write the tile-pair interleaved layout (tiles_ilv_ok said yes)
int run_fwd_pass(int pass, const FwdDesc *jd, int njobs, int jobs_per_cta, cudaStream_t s, int ilv = 0)
{
    const Plan &sh = *jd[0].pl;
    const int l0 = sh.pass_l0[pass], l1 = sh.pass_l1[pass];
    ColFwdParams CP;
    if (fwd_params(pass, jd, njobs, jobs_per_cta, CP)) {
        CP.ilv = ilv;
        FCIRC_TRY(fwd_tma_maps(CP, njobs, l1 - l0));
        return launch_colfwd(CP, njobs / jobs_per_cta, s);
    }
    if (ilv) return fail(FCIRC_EINVAL, "interleaved layout requested from a strided pass");
    StrFwdParams P{};
    for (int k = 0; k < njobs; ++k)
        P.job[k] = StrFwdJob{jd[k].src, jd[k].dst, jd[k].pl->d_ftw, jd[k].pl->p, jd[k].vec_side};
    P.N = sh.n;
    P.logn = sh.m;
    P.l0 = l0;
    P.l1 = l1;
    P.logW = 2;
    return launch_strided_fwd(P, njobs, s);
}

struct InvDesc {
    const uint32_t *src;
    uint32_t *dst;
    const Plan *pl;
};

bool inv_params(int pass, const InvDesc *jd, int nprime, int epi, uint64_t *dst64, uint64_t nout,
                const CrtConsts *crt, ColInvParams &P)
{
    const Plan &sh = *jd[0].pl;
    const int l0 = sh.pass_l0[pass], l1 = sh.pass_l1[pass];
    if (!fast_col_ok(l1 - l0, sh.m - l1)) return false;
    P = ColInvParams{};
    for (int q = 0; q < nprime; ++q)
        P.job[q] = ColInvJob{jd[q].src, jd[q].dst, jd[q].pl->d_gitw + jd[q].pl->pass_goff[pass], jd[q].pl->p,
                             jd[q].pl->d_gitwl + jd[q].pl->pass_loff[pass]};
    P.nprime = nprime;
    P.N = (uint32_t)sh.n;
    P.logn = sh.m;
    P.l0 = l0;
    P.l1 = l1;
    for (int st = 0; st < 3; ++st) P.stage_off[st] = sh.stage_off[pass][st];
    P.epi = epi;
    P.dst64 = dst64;
    P.nout = nout;
    if (crt) P.crt = *crt;
    return true;
}

// ilv: read the tile-pair interleaved layout (tiles_ilv_ok said yes)
int run_inv_pass(int pass, const InvDesc *jd, int nprime, int epi, uint64_t *dst64, uint64_t nout,
                 const CrtConsts *crt, cudaStream_t s, int ilv = 0)
{
    const Plan &sh = *jd[0].pl;
    const int l0 = sh.pass_l0[pass], l1 = sh.pass_l1[pass];
    ColInvParams CP;
    if (inv_params(pass, jd, nprime, epi, dst64, nout, crt, CP)) {
        CP.ilv = ilv;
        return launch_colinv(CP, s);
    }
    if (ilv) return fail(FCIRC_EINVAL, "interleaved layout requested from a strided pass");
    StrInvParams P{};
    for (int q = 0; q < nprime; ++q) P.job[q] = StrInvJob{jd[q].src, jd[q].dst, jd[q].pl->d_fitw, jd[q].pl->p};
    P.nprime = nprime;
    P.N = sh.n;
    P.logn = sh.m;
    P.l0 = l0;
    P.l1 = l1;
    P.logW = 2;
    P.epi = epi;
    P.dst64 = dst64;
    P.nout = nout;
    if (crt) P.crt = *crt;
    return launch_strided_inv(P, s);
}

Src src_u32(const void *ptr, uint64_t n) { return Src{ptr, n, SRC_U32, 0, Tw{0, 0}}; }

// Whether the arrays between the last forward column pass, the 4096-residue
// tiles and the first inverse column pass can take the tile-pair interleaved
// layout (ilv_pos): the four-column kernels run both passes and the tile
// kernel is the register-staged one.  `fwd` and `inv` describe the last
// forward pass (index npass - 1) and the first inverse pass (the same index).
bool tiles_ilv_ok(const Plan &pl, const FwdDesc *fwd, int njobs, int jobs_per_cta, const InvDesc *inv, int nprime,
                  int epi, uint64_t *dst64, uint64_t nout, const CrtConsts *crt)
{
    if (pl.k == 0 || pl.npass < 1 || !fast_tile_ok(pl.logT)) return false;
    ColFwdParams F;
    ColInvParams I;
    const int last = pl.npass - 1;
    if (!fwd_params(last, fwd, njobs, jobs_per_cta, F) || !inv_params(last, inv, nprime, epi, dst64, nout, crt, I))
        return false;
    // an interleaved array cannot be recombined in place: the natural
    // positions a column group writes hold interleaved residues of other
    // column groups, which other CTAs may not have read yet
    if (!epi_crt(epi))
        for (int q = 0; q < nprime; ++q)
            if (inv[q].src == inv[q].dst) return false;
    return col4_fwd_ilv_ok(F, njobs / jobs_per_cta) && col4_inv_ilv_ok(I);
}

}  // namespace

// The f-circulant product c = A x for n >= 2 with the plan pl: row vector
// source sa (scaled by 2^32 2^-L on its first load), vector source sx, the
// row side worked in c itself, the vector side in xs (n words, used when the
// column passes run).  Canonical output.
static int matvec_core(const Plan *pl, const Src &sa, const Src &sx, uint32_t *dc, uint32_t *xs, cudaStream_t s)
{
    const uint64_t n = pl->n;
    if (pl->k == 0) {
        TileParams tp;
        tp.job[0] = tile_job(pl, sa, sx, dc, 0);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        return run_tile(tp, 1, 1, s);
    }
    auto fwd_desc = [&](int i, FwdDesc *jd) {
        jd[0] = FwdDesc{i == 0 ? sa : src_u32(dc, n), dc, pl, 0, 0};
        jd[1] = FwdDesc{i == 0 ? sx : src_u32(xs, n), xs, pl, 1, 0};
    };
    // the tiles leave their products in xs; the first recombination pass
    // reads them there and writes c, the others work in place in c
    const int last = pl->npass - 1;
    auto inv_desc = [&](int i) { return InvDesc{i == last ? xs : dc, dc, pl}; };
    FwdDesc ljd[2];
    fwd_desc(last, ljd);
    const InvDesc lid[1] = {inv_desc(last)};
    const int ilv = tiles_ilv_ok(*pl, ljd, 2, 1, lid, 1, last == 0 ? EPI_CANON : EPI_LAZY, nullptr, 0, nullptr);
    for (int i = 0; i < pl->npass; ++i) {
        FwdDesc jd[2];
        fwd_desc(i, jd);
        FCIRC_TRY(run_fwd_pass(i, jd, 2, 1, s, i == last ? ilv : 0));
    }
    {
        TileParams tp;
        tp.job[0] = tile_job(pl, src_u32(dc, n), src_u32(xs, n), xs, 1);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        tp.ilv = ilv ? 3 : 0;
        FCIRC_TRY(tile_tma_maps(tp, 1));
        FCIRC_TRY(run_tile(tp, (uint64_t)1 << pl->k, 1, s));
    }
    for (int i = last; i >= 0; --i) {
        const InvDesc jd[1] = {inv_desc(i)};
        FCIRC_TRY(run_inv_pass(i, jd, 1, i == 0 ? EPI_CANON : EPI_LAZY, nullptr, 0, nullptr, s, i == last ? ilv : 0));
    }
    return FCIRC_OK;
}

// Corollary 1: an n x n product with n not a power of two (f-circulant with
// row vector a, or Toeplitz with diagonals t[0 .. 2n-2]) as the first n
// entries of an ordinary circulant product of size N >= 2n - 1 (a power of
// two), built by k_embed.  `a` holds n (f-circulant) or 2n - 1 (Toeplitz)
// words.
static int embedded_matvec(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x, uint32_t *c, uint64_t n,
                           int toeplitz, cudaStream_t s)
{
    uint64_t N = 2;
    while (N < 2 * n - 1) N <<= 1;
    if (N > ((uint64_t)1 << kMaxLogN)) return fail(FCIRC_EINVAL, "n = %llu needs an embedding above 2^%d",
                                                   (unsigned long long)n, kMaxLogN);
    const PrimeTables *pt;
    FCIRC_TRY(prime_tables(p, &pt));
    const Plan *pl = nullptr;
    FCIRC_TRY(get_plan(p, 1, N, &pl));
    const uint64_t na = toeplitz ? 2 * n - 1 : n;
    Arg aa{a, na * 4, true, false}, ax{x, n * 4, true, false}, ac{c, n * 4, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, 4 * N * 4));
    const uint32_t *da = static_cast<const uint32_t *>(aa.d), *dx = static_cast<const uint32_t *>(ax.d);
    FCIRC_TRY(check_lt(da, na, p, s));
    FCIRC_TRY(check_lt(dx, n, p, s));
    uint32_t *ap = reinterpret_cast<uint32_t *>(st.scratch), *bp = ap + N, *cp = bp + N, *xs = cp + N;
    const uint32_t fr = f % p;
    FCIRC_TRY(launch_embed(toeplitz ? da + (n - 1) : da, da, dx, n, N, Tw{fr, host::shoup_quot(fr, p)}, p,
                           toeplitz, ap, bp, s));
    FCIRC_TRY(matvec_core(pl, Src{ap, N, SRC_U32, 1, pl->kt}, src_u32(bp, N), cp, xs, s));
    FCIRC_CUDA_TRY(cudaMemcpyAsync(ac.d, cp, n * 4, cudaMemcpyDeviceToDevice, s));
    return st.end();
}

// The three NTT-friendly primes of the polynomial and large-integer
// products (2^23, 2^26 and 2^25 divide p - 1; their product exceeds 2^85).
static const uint32_t kPrimes[3] = {998244353u, 469762049u, 167772161u};

// Product of 16-bit coefficient vectors as residues mod the three primes,
// recombined by CRT into 64-bit columns: the shared core of poly_mul_int and
// bigint_mul.  P, Q, out are device pointers; `scratch` has
// poly_scratch_bytes(N) bytes.
static size_t poly_scratch_bytes(uint64_t N) { return (size_t)6 * N * 4; }

static int poly_core(const uint16_t *P, uint64_t np, const uint16_t *Q, uint64_t nq, uint64_t *out,
                     uint64_t nout, uint64_t N, char *scratch, cudaStream_t s)
{
    const Plan *pl[3];
    for (int q = 0; q < 3; ++q) FCIRC_TRY(get_plan(kPrimes[q], 1, N, &pl[q]));
    const CrtConsts crt = make_crt(kPrimes[0], kPrimes[1], kPrimes[2]);
    uint32_t *A[3], *X[3];
    for (int q = 0; q < 3; ++q) {
        A[q] = reinterpret_cast<uint32_t *>(scratch) + (size_t)q * N;
        X[q] = reinterpret_cast<uint32_t *>(scratch) + (size_t)(3 + q) * N;
    }
    // row vector: P reversed (a'[i] = P[N-1-i]) and scaled by 2^32 2^-L for
    // the leaf; vector: Q; both zero-padded to N
    Src srcP[3], srcQ{Q, nq, SRC_U16, 0, Tw{0, 0}};
    for (int q = 0; q < 3; ++q) srcP[q] = Src{P, np, SRC_U16_REV, 1, pl[q]->kt};
    const Plan &p0 = *pl[0];
    if (p0.k == 0) {
        TileParams tp;
        for (int q = 0; q < 3; ++q) tp.job[q] = tile_job(pl[q], srcP[q], srcQ, A[q], 0);
        tp.N = N;
        tp.logT = p0.logT;
        tp.D = p0.D;
        FCIRC_TRY(run_tile(tp, 1, 3, s));
        return launch_crt_rot(A[0], A[1], A[2], N, out, nout, crt, s);
    }
    auto fwd_desc = [&](int i, FwdDesc *jd) {
        // f = 1 gives s = 1 at level 0; with both inputs shorter than N/2 that
        // level only copies (row vector zero below N/2, vector from N/2)
        const int half = (np <= N / 2 && nq <= N / 2) ? 1 : 0;
        for (int q = 0; q < 3; ++q) {
            if (i == 0) {
                jd[q] = FwdDesc{srcP[q], A[q], pl[q], 0, half};
                jd[3 + q] = FwdDesc{srcQ, X[q], pl[q], 1, 2 * half};
            } else {
                jd[q] = FwdDesc{src_u32(A[q], N), A[q], pl[q], 0, 0};
                jd[3 + q] = FwdDesc{src_u32(X[q], N), X[q], pl[q], 1, 0};
            }
        }
    };
    // The reversed-row embedding moves the product up by one entry
    // (coefficient k is circulant entry k + 1).  The 4096-residue tile kernel
    // undoes that in its leaves (TILE_SHIFT: the row vector shifted by one
    // place, an identity at f = 1), so the CRT writes whole aligned sectors;
    // the other tile kernels leave it to the CRT (EPI_CRT_ROT).
    const bool shift = fast_tile_ok(p0.logT);
    InvDesc ijd[3];
    for (int q = 0; q < 3; ++q) ijd[q] = InvDesc{A[q], A[q], pl[q]};
    const int last = p0.npass - 1;
    auto epi_of = [&](int i) { return i == 0 ? (shift ? EPI_CRT : EPI_CRT_ROT) : EPI_LAZY; };
    FwdDesc ljd[6];
    fwd_desc(last, ljd);
    const int ilv = tiles_ilv_ok(p0, ljd, 6, 3, ijd, 3, epi_of(last), out, nout, &crt);
    for (int i = 0; i < p0.npass; ++i) {
        FwdDesc jd[6];
        fwd_desc(i, jd);
        FCIRC_TRY(run_fwd_pass(i, jd, 6, 3, s, i == last ? ilv : 0));
    }
    {
        TileParams tp;
        for (int q = 0; q < 3; ++q) tp.job[q] = tile_job(pl[q], src_u32(A[q], N), src_u32(X[q], N), A[q], 1);
        tp.N = N;
        tp.logT = p0.logT;
        tp.D = p0.D;
        tp.var = shift ? TILE_SHIFT : TILE_FULL;
        tp.ilv = ilv ? 3 : 0;
        FCIRC_TRY(tile_tma_maps(tp, 3));
        FCIRC_TRY(run_tile(tp, (uint64_t)1 << p0.k, 3, s));
    }
    for (int i = last; i >= 0; --i)
        FCIRC_TRY(run_inv_pass(i, ijd, 3, epi_of(i), out, nout, &crt, s, i == last ? ilv : 0));
    return FCIRC_OK;
}

}  // namespace fcirc

using namespace fcirc;

extern "C" {

const char *fcirc_error_string(int status)
{
    switch (status) {
    case FCIRC_OK: return "FCIRC_OK";
    case FCIRC_EINVAL: return "FCIRC_EINVAL: invalid argument";
    case FCIRC_ENOROOT: return "FCIRC_ENOROOT: a root required by Theorem 1 does not exist";
    case FCIRC_ENOMEM: return "FCIRC_ENOMEM: device allocation failed";
    case FCIRC_ECUDA: return "FCIRC_ECUDA: CUDA runtime error";
    case FCIRC_ETIMEOUT: return "FCIRC_ETIMEOUT: a bounded device wait gave up";
    default: return "unknown fcirc status";
    }
}

const char *fcirc_last_error(void) { return last_error_detail(); }

int fcirc_matvec(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x, uint32_t *c,
                 uint64_t n, void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec: null pointer");
    if (n == 0) return fail(FCIRC_EINVAL, "fcirc_matvec: n = 0");
    // n not a power of two: Corollary 1
    if (!is_pow2(n)) return embedded_matvec(p, f, a, x, c, n, 0, static_cast<cudaStream_t>(stream));
    if (n > ((uint64_t)1 << kMaxLogN)) return fail(FCIRC_EINVAL, "fcirc_matvec: n above 2^%d", kMaxLogN);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Plan *pl = nullptr;
    if (n == 1) {
        const PrimeTables *pt;
        FCIRC_TRY(prime_tables(p, &pt));
        if (f % p == 0) return fail(FCIRC_ENOROOT, "f = 0 has no inverse (Theorem 1)");
    } else {
        FCIRC_TRY(get_plan(p, f, n, &pl));
    }
    Arg aa{a, n * 4, true, false}, ax{x, n * 4, true, false}, ac{c, n * 4, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    const size_t extra = (pl && pl->k > 0) ? n * 4 : 0;
    FCIRC_TRY(st.begin(s, extra));
    const uint32_t *da = static_cast<const uint32_t *>(aa.d), *dx = static_cast<const uint32_t *>(ax.d);
    uint32_t *dc = static_cast<uint32_t *>(ac.d);
    if (n == 1) {
        FCIRC_TRY(launch_scalar(da, dx, dc, p, s));
        return st.end();
    }
    FCIRC_TRY(check_lt(da, n, p, s));
    FCIRC_TRY(check_lt(dx, n, p, s));
    // the row vector is scaled by 2^32 2^-L on its first load (see leaf2)
    const Src sa{da, n, SRC_U32, 1, pl->kt};
    FCIRC_TRY(matvec_core(pl, sa, src_u32(dx, n), dc, reinterpret_cast<uint32_t *>(st.scratch), s));
    return st.end();
}

int fcirc_toeplitz_matvec(uint32_t p, const uint32_t *t, const uint32_t *x, uint32_t *c, uint64_t n, void *stream)
{
    set_error("");
    if (!t || !x || !c) return fail(FCIRC_EINVAL, "fcirc_toeplitz_matvec: null pointer");
    if (n == 0) return fail(FCIRC_EINVAL, "fcirc_toeplitz_matvec: n = 0");
    return embedded_matvec(p, 0, t, x, c, n, 1, static_cast<cudaStream_t>(stream));
}

int fcirc_matvec_t(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x, uint32_t *c, uint64_t n,
                   void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_t: null pointer");
    if (!is_pow2(n)) return fail(FCIRC_EINVAL, "fcirc_matvec_t: n = %llu is not a power of two",
                                 (unsigned long long)n);
    if (n > ((uint64_t)1 << kMaxLogN)) return fail(FCIRC_EINVAL, "fcirc_matvec_t: n above 2^%d", kMaxLogN);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PrimeTables *pt;
    FCIRC_TRY(prime_tables(p, &pt));
    if (f % p == 0) return fail(FCIRC_ENOROOT, "f = 0 has no inverse (Theorem 1)");
    // A^T x = the row product with parameter f^-1 of the reversed row vector,
    // rotated by one and scaled by f (all but its first element)
    const uint32_t fi = host::invmod(f % p, p);
    const Plan *pl = nullptr;
    if (n > 1) FCIRC_TRY(get_plan(p, fi, n, &pl));
    Arg aa{a, n * 4, true, false}, ax{x, n * 4, true, false}, ac{c, n * 4, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, 2 * n * 4));
    const uint32_t *da = static_cast<const uint32_t *>(aa.d), *dx = static_cast<const uint32_t *>(ax.d);
    uint32_t *dc = static_cast<uint32_t *>(ac.d);
    if (n == 1) {
        FCIRC_TRY(launch_scalar(da, dx, dc, p, s));
        return st.end();
    }
    FCIRC_TRY(check_lt(da, n, p, s));
    FCIRC_TRY(check_lt(dx, n, p, s));
    uint32_t *cr = reinterpret_cast<uint32_t *>(st.scratch), *xs = cr + n;
    const Src sa{da, n, SRC_U32_REV, 1, pl->kt};
    FCIRC_TRY(matvec_core(pl, sa, src_u32(dx, n), cr, xs, s));
    FCIRC_TRY(launch_rot_scale(cr, dc, n, Tw{f % p, host::shoup_quot(f % p, p)}, p, s));
    return st.end();
}

// -- fixed-matrix plans ----------------------------------------------------------

}  // extern "C"

struct fcirc_aplan {
    uint32_t p, f;
    uint64_t n;
    int dev;
    const Plan *pl;     // nullptr when n == 1
    uint32_t *ahat;     // transformed row vector (planned) or the row vector itself
    bool planned;       // n >= 4096: products run two of the three trees
};

extern "C" {

int fcirc_aplan_create(uint32_t p, uint32_t f, const uint32_t *a, uint64_t n, void *stream, fcirc_aplan_t *out)
{
    set_error("");
    if (!out) return fail(FCIRC_EINVAL, "fcirc_aplan_create: null plan pointer");
    *out = nullptr;
    if (!a) return fail(FCIRC_EINVAL, "fcirc_aplan_create: null pointer");
    if (!is_pow2(n)) return fail(FCIRC_EINVAL, "fcirc_aplan_create: n = %llu is not a power of two",
                                 (unsigned long long)n);
    if (n > ((uint64_t)1 << kMaxLogN)) return fail(FCIRC_EINVAL, "fcirc_aplan_create: n above 2^%d", kMaxLogN);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Plan *pl = nullptr;
    if (n == 1) {
        const PrimeTables *pt;
        FCIRC_TRY(prime_tables(p, &pt));
        if (f % p == 0) return fail(FCIRC_ENOROOT, "f = 0 has no inverse (Theorem 1)");
    } else {
        FCIRC_TRY(get_plan(p, f, n, &pl));
    }
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    void *mem = nullptr;
    if (dev_alloc(&mem, n * 4) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(FCIRC_ENOMEM, "fcirc_aplan_create: %llu bytes of device memory", (unsigned long long)(n * 4));
    }
    fcirc_aplan *h = new fcirc_aplan{p, f % p, n, dev, pl, static_cast<uint32_t *>(mem), false};
    auto undo = [&](int st) {
        cudaFree(mem);
        delete h;
        return st;
    };
    Arg aa{a, n * 4, true, false};
    Staging st;
    st.args = {&aa};
    int rc = st.begin(s, 0);
    if (rc != FCIRC_OK) return undo(rc);
    const uint32_t *da = static_cast<const uint32_t *>(aa.d);
    rc = check_lt(da, n, p, s);
    if (rc != FCIRC_OK) return undo(rc);
    h->planned = pl && pl->logT == 12;
    if (!h->planned) {
        if (cudaMemcpyAsync(h->ahat, da, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return undo(fail(FCIRC_ECUDA, "fcirc_aplan_create: copy of the row vector"));
    } else {
        // the row vector's tree: the forward column passes of the row side,
        // then the tiles' row levels (scaled by 2^32 2^-L on the first load)
        const Src sa{da, n, SRC_U32, 1, pl->kt};
        for (int i = 0; i < pl->npass; ++i) {
            FwdDesc jd[1] = {FwdDesc{i == 0 ? sa : src_u32(h->ahat, n), h->ahat, pl, 0, 0}};
            rc = run_fwd_pass(i, jd, 1, 1, s);
            if (rc != FCIRC_OK) return undo(rc);
        }
        TileParams tp;
        tp.job[0] = tile_job(pl, pl->k == 0 ? sa : src_u32(h->ahat, n), src_u32(h->ahat, n), h->ahat, 1);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        tp.var = TILE_ROW;
        rc = run_tile(tp, (uint64_t)1 << pl->k, 1, s);
        if (rc != FCIRC_OK) return undo(rc);
    }
    rc = st.end();
    if (rc != FCIRC_OK) return undo(rc);
    *out = h;
    return FCIRC_OK;
}

int fcirc_matvec_aplan(fcirc_aplan_t h, const uint32_t *x, uint32_t *c, void *stream)
{
    set_error("");
    if (!h) return fail(FCIRC_EINVAL, "fcirc_matvec_aplan: null plan");
    if (!x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_aplan: null pointer");
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h->dev)
        return fail(FCIRC_EINVAL, "fcirc_matvec_aplan: plan lives on device %d, current device is %d", h->dev, dev);
    if (!h->planned) return fcirc_matvec(h->p, h->f, h->ahat, x, c, h->n, stream);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n = h->n;
    const Plan *pl = h->pl;
    Arg ax{x, n * 4, true, false}, ac{c, n * 4, false, true};
    Staging st;
    st.args = {&ax, &ac};
    FCIRC_TRY(st.begin(s, pl->k > 0 ? n * 4 : 0));
    const uint32_t *dx = static_cast<const uint32_t *>(ax.d);
    uint32_t *dc = static_cast<uint32_t *>(ac.d);
    FCIRC_TRY(check_lt(dx, n, h->p, s));
    const Src sx = src_u32(dx, n), sah = src_u32(h->ahat, n);
    if (pl->k == 0) {
        TileParams tp;
        tp.job[0] = tile_job(pl, sah, sx, dc, 0);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        tp.var = TILE_PLANNED;
        FCIRC_TRY(run_tile(tp, 1, 1, s));
        return st.end();
    }
    // the vector's tree in the scratch, the tiles (transformed row vector
    // read as it is) in place there, and the recombination into c
    // (the vector side and the tile output may take the interleaved layout;
    // the transformed row vector keeps the tile kernel's own layout)
    uint32_t *xs = reinterpret_cast<uint32_t *>(st.scratch);
    const int last = pl->npass - 1;
    auto fjd = [&](int i) { return FwdDesc{i == 0 ? sx : src_u32(xs, n), xs, pl, 1, 0}; };
    // the first recombination pass reads the tiles' products in xs and
    // writes c; the others work in place in c
    auto ijd = [&](int i) { return InvDesc{i == last ? xs : dc, dc, pl}; };
    const FwdDesc lf[1] = {fjd(last)};
    const InvDesc li[1] = {ijd(last)};
    const int ilv = tiles_ilv_ok(*pl, lf, 1, 1, li, 1, last == 0 ? EPI_CANON : EPI_LAZY, nullptr, 0, nullptr);
    for (int i = 0; i < pl->npass; ++i) {
        FwdDesc jd[1] = {fjd(i)};
        FCIRC_TRY(run_fwd_pass(i, jd, 1, 1, s, i == last ? ilv : 0));
    }
    {
        TileParams tp;
        tp.job[0] = tile_job(pl, sah, src_u32(xs, n), xs, 1);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        tp.var = TILE_PLANNED;
        tp.ilv = ilv ? 2 : 0;
        FCIRC_TRY(tile_tma_maps(tp, 1));
        FCIRC_TRY(run_tile(tp, (uint64_t)1 << pl->k, 1, s));
    }
    for (int i = last; i >= 0; --i) {
        InvDesc jd[1] = {ijd(i)};
        FCIRC_TRY(run_inv_pass(i, jd, 1, i == 0 ? EPI_CANON : EPI_LAZY, nullptr, 0, nullptr, s,
                               i == last ? ilv : 0));
    }
    return st.end();
}

int fcirc_aplan_destroy(fcirc_aplan_t h)
{
    set_error("");
    if (!h) return FCIRC_OK;
    int cur = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->dev) FCIRC_CUDA_TRY(cudaSetDevice(h->dev));
    const cudaError_t e = cudaFree(h->ahat);
    if (cur != h->dev) (void)cudaSetDevice(cur);
    delete h;
    if (e != cudaSuccess) return fail(FCIRC_ECUDA, "fcirc_aplan_destroy: %s", cudaGetErrorString(e));
    return FCIRC_OK;
}

int poly_mul_int(const uint16_t *P, uint64_t np, const uint16_t *Q, uint64_t nq, int64_t *out,
                 void *stream)
{
    set_error("");
    if (!P || !Q || !out) return fail(FCIRC_EINVAL, "poly_mul_int: null pointer");
    if (np == 0 || nq == 0) return fail(FCIRC_EINVAL, "poly_mul_int: empty polynomial");
    const uint64_t nout = np + nq - 1;
    if (nout > ((uint64_t)1 << 24))
        return fail(FCIRC_EINVAL, "poly_mul_int: np + nq - 1 = %llu exceeds 2^24",
                    (unsigned long long)nout);
    uint64_t N = 2;
    while (N < nout) N <<= 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // plans first: they may allocate and synchronise
    for (int q = 0; q < 3; ++q) {
        const Plan *pl;
        FCIRC_TRY(get_plan(kPrimes[q], 1, N, &pl));
    }
    Arg aP{P, np * 2, true, false}, aQ{Q, nq * 2, true, false}, aO{out, nout * 8, false, true};
    Staging st;
    st.args = {&aP, &aQ, &aO};
    FCIRC_TRY(st.begin(s, poly_scratch_bytes(N)));
    FCIRC_TRY(poly_core(static_cast<const uint16_t *>(aP.d), np, static_cast<const uint16_t *>(aQ.d), nq,
                        static_cast<uint64_t *>(aO.d), nout, N, st.scratch, s));
    return st.end();
}

int bigint_mul(const uint16_t *A, uint64_t na, const uint16_t *B, uint64_t nb, uint16_t *out, void *stream)
{
    set_error("");
    if (!A || !B || !out) return fail(FCIRC_EINVAL, "bigint_mul: null pointer");
    if (na == 0 || nb == 0) return fail(FCIRC_EINVAL, "bigint_mul: empty operand");
    const uint64_t ncols = na + nb - 1, nlimbs = na + nb;
    if (ncols > ((uint64_t)1 << 24))
        return fail(FCIRC_EINVAL, "bigint_mul: na + nb - 1 = %llu exceeds 2^24 limbs", (unsigned long long)ncols);
    uint64_t N = 2;
    while (N < ncols) N <<= 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int q = 0; q < 3; ++q) {
        const Plan *pl;
        FCIRC_TRY(get_plan(kPrimes[q], 1, N, &pl));
    }
    Arg aA{A, na * 2, true, false}, aB{B, nb * 2, true, false}, aO{out, nlimbs * 2, false, true};
    Staging st;
    st.args = {&aA, &aB, &aO};
    // scratch: the polynomial pipeline, the 64-bit column sums, the carry maps
    const size_t pb = (poly_scratch_bytes(N) + 255) & ~(size_t)255;
    const size_t cb = (ncols * 8 + 255) & ~(size_t)255;
    FCIRC_TRY(st.begin(s, pb + cb + carry_scratch_bytes(nlimbs)));
    uint64_t *cols = reinterpret_cast<uint64_t *>(st.scratch + pb);
    // column sums sum_{i+j=k} A_i B_j: the polynomial product of the limb
    // vectors (Section 3.2: the parts as polynomial coefficients)
    FCIRC_TRY(poly_core(static_cast<const uint16_t *>(aA.d), na, static_cast<const uint16_t *>(aB.d), nb, cols,
                        ncols, N, st.scratch, s));
    FCIRC_TRY(launch_carry(cols, ncols, static_cast<uint16_t *>(aO.d), nlimbs, st.scratch + pb + cb, s));
    return st.end();
}

int fcirc_matvec_c64(const float *a, const float *x, float *c, double f_re, double f_im, uint64_t n,
                     uint64_t batch, void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_c64: null pointer");
    if (!is_pow2(n) || n < 8 || n > 4096)
        return fail(FCIRC_EINVAL, "fcirc_matvec_c64: n = %llu must be a power of two in [8, 4096]",
                    (unsigned long long)n);
    if (f_re == 0.0 && f_im == 0.0) return fail(FCIRC_ENOROOT, "fcirc_matvec_c64: f = 0 has no inverse");
    if (batch == 0) return FCIRC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = ilog2(n);
    CParams P{};
    FCIRC_TRY(complex_tables(f_re, f_im, n, &P.tw, &P.itw));
    const size_t bytes = n * batch * 8;
    Arg aa{a, bytes, true, false}, ax{x, bytes, true, false}, ac{c, bytes, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, 0));
    P.a = static_cast<const float *>(aa.d);
    P.x = static_cast<const float *>(ax.d);
    P.c = static_cast<float *>(ac.d);
    P.batch = batch;
    P.scale = std::ldexp(1.0f, -(m - 1));
    FCIRC_TRY(launch_cfwd(P, m, s));
    return st.end();
}

int fcirc_matvec_gf(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t f_re, uint32_t f_im, uint64_t n,
                    uint64_t batch, void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_gf: null pointer");
    if (!is_pow2(n) || n < 8 || n > 4096)
        return fail(FCIRC_EINVAL, "fcirc_matvec_gf: n = %llu must be a power of two in [8, 4096]",
                    (unsigned long long)n);
    if (f_re >= gf::P || f_im >= gf::P) return fail(FCIRC_EINVAL, "fcirc_matvec_gf: f not canonical");
    if (f_re == 0 && f_im == 0) return fail(FCIRC_ENOROOT, "fcirc_matvec_gf: f = 0 has no inverse");
    if (batch == 0) return FCIRC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = ilog2(n);
    GParams P{};
    FCIRC_TRY(gf_tables(f_re, f_im, n, &P.tw, &P.itw));
    const size_t bytes = n * batch * 8;
    Arg aa{a, bytes, true, false}, ax{x, bytes, true, false}, ac{c, bytes, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, 0));
    P.a = static_cast<const uint32_t *>(aa.d);
    P.x = static_cast<const uint32_t *>(ax.d);
    P.c = static_cast<uint32_t *>(ac.d);
    P.batch = batch;
    P.scale = gf::inv(gf::E{(uint32_t)1u << (m - 1), 0u}).re;   // 2^-L, L = m - 1
    FCIRC_TRY(check_lt(P.a, 2 * n * batch, gf::P, s));
    FCIRC_TRY(check_lt(P.x, 2 * n * batch, gf::P, s));
    FCIRC_TRY(launch_gfwd(P, m, s));
    return st.end();
}

int fcirc_matvec_ssa(const uint64_t *a, const uint64_t *x, uint64_t *c, uint32_t K, uint32_t f_exp, uint64_t n,
                     uint64_t batch, void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_ssa: null pointer");
    if (K != 64 && K != 128) return fail(FCIRC_EINVAL, "fcirc_matvec_ssa: K = %u (64 or 128)", K);
    if (!is_pow2(n) || n < 8 || n > 512 || n > 4ull * K)
        return fail(FCIRC_EINVAL, "fcirc_matvec_ssa: n = %llu must be a power of two in [8, min(512, 4K)]",
                    (unsigned long long)n);
    if (f_exp >= 2 * K) return fail(FCIRC_EINVAL, "fcirc_matvec_ssa: f = 2^%u with the exponent above 2K", f_exp);
    if (batch == 0) return FCIRC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = ilog2(n), L = m - 1;
    SParams P{};
    FCIRC_TRY(ssa_tables(K, f_exp, n, &P.tw, &P.itw));
    const size_t bytes = n * batch * (K / 64 + 1) * 8;
    Arg aa{a, bytes, true, false}, ax{x, bytes, true, false}, ac{c, bytes, false, true};
    Staging st;
    st.args = {&aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, 0));
    P.a = static_cast<const uint64_t *>(aa.d);
    P.x = static_cast<const uint64_t *>(ax.d);
    P.c = static_cast<uint64_t *>(ac.d);
    P.batch = batch;
    P.scale_exp = (int)((2 * K - L) % (2 * K));
    FCIRC_TRY(launch_sfwd(P, (int)K, m, s));
    return st.end();
}

int fcirc_matvec_backward(const float *a, const float *x, const float *g, double f_re, double f_im,
                          float *grad_a, float *grad_x, uint64_t n, uint64_t batch, void *stream)
{
    set_error("");
    if (!a || !x || !g || !grad_a || !grad_x) return fail(FCIRC_EINVAL, "fcirc_matvec_backward: null pointer");
    if (!is_pow2(n) || n < 8 || n > 4096)
        return fail(FCIRC_EINVAL, "fcirc_matvec_backward: n = %llu must be a power of two in [8, 4096]",
                    (unsigned long long)n);
    const double f2 = f_re * f_re + f_im * f_im;
    if (f2 == 0.0) return fail(FCIRC_ENOROOT, "fcirc_matvec_backward: f = 0 has no inverse");
    if (batch == 0) return FCIRC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int m = ilog2(n);
    CBwdParams P{};
    // dL/dx: parameter 1/conj(f) = f / |f|^2; dL/da: parameter conj(f)
    FCIRC_TRY(complex_tables(f_re / f2, f_im / f2, n, &P.tw_x, &P.itw_x));
    FCIRC_TRY(complex_tables(f_re, -f_im, n, &P.tw_a, &P.itw_a));
    const size_t bytes = n * batch * 8;
    Arg aa{a, bytes, true, false}, ax{x, bytes, true, false}, ag{g, bytes, true, false};
    Arg oa{grad_a, bytes, false, true}, ox{grad_x, bytes, false, true};
    Staging st;
    st.args = {&aa, &ax, &ag, &oa, &ox};
    FCIRC_TRY(st.begin(s, 0));
    P.a = static_cast<const float *>(aa.d);
    P.x = static_cast<const float *>(ax.d);
    P.g = static_cast<const float *>(ag.d);
    P.grad_a = static_cast<float *>(oa.d);
    P.grad_x = static_cast<float *>(ox.d);
    P.fc_re = (float)f_re;
    P.fc_im = (float)(-f_im);
    P.batch = batch;
    P.scale = std::ldexp(1.0f, -(m - 1));
    FCIRC_TRY(launch_cbwd(P, m, s));
    return st.end();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched products: configurations, autotuner cache, graph handles

namespace fcirc {
namespace {

// Tunable launch shapes of the batched kernel: persistent CTAs per SM, and
// the tile size (levels per in-CTA pass follow from it) for large instances.
struct BConfig {
    int ctas_per_sm;
    int big_log;
};
const BConfig kBConfigs[] = {{1, 12}, {2, 12}, {3, 12}, {4, 12}, {1, 11}, {2, 11}, {3, 11}, {4, 11}};
constexpr int kNumBConfigs = sizeof(kBConfigs) / sizeof(kBConfigs[0]);
constexpr int kDefaultBConfig = 3;   // four CTAs per SM, 4096-residue tiles: the tuner's choice on GB300

std::mutex g_tune_mu;
std::map<std::tuple<int, uint32_t, uint32_t, uint64_t>, int> g_tune;   // (dev, p, count, total) -> config
bool g_tune_loaded = false;

const char *tune_path() { return std::getenv("FCIRC_TUNE_CACHE"); }

void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = tune_path();
    if (!path) return;
    FILE *fh = fopen(path, "r");
    if (!fh) return;
    int dev, cfg;
    unsigned p, count;
    unsigned long long total;
    while (fscanf(fh, "%d %u %u %llu %d", &dev, &p, &count, &total, &cfg) == 5)
        if (cfg >= 0 && cfg < kNumBConfigs) g_tune[{dev, p, count, (uint64_t)total}] = cfg;
    fclose(fh);
}

void tune_store_locked()
{
    const char *path = tune_path();
    if (!path) return;
    FILE *fh = fopen(path, "w");
    if (!fh) return;
    for (auto &kv : g_tune)
        fprintf(fh, "%d %u %u %llu %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                (unsigned long long)std::get<3>(kv.first), kv.second);
    fclose(fh);
}

int tuned_config(uint32_t p, uint32_t count, uint64_t total)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find({dev, p, count, total});
    return it == g_tune.end() ? kDefaultBConfig : it->second;
}

// Everything a batched launch needs except the per-call pointers.
int batch_setup(uint32_t p, uint32_t count, uint64_t total, BatchParams &P)
{
    const PrimeTables *pt;
    FCIRC_TRY(prime_tables(p, &pt));
    P.p = p;
    P.pinv = pt->pinv;
    P.Om = pt->omega;
    P.v = pt->v;
    P.U = pt->d_U;
    P.Ui = pt->d_Ui;
    P.count = count;
    P.total = total;
    FCIRC_TRY(device_status_word(&P.status));
    return FCIRC_OK;
}

int launch_with_config(BatchParams P, int cfg, cudaStream_t s)
{
    const BConfig &c = kBConfigs[cfg];
    int maxc = batch_max_ctas_per_sm();
    if (maxc <= 0) maxc = 1;
    P.big_log = c.big_log;
    const int cps = c.ctas_per_sm < maxc ? c.ctas_per_sm : maxc;
    return launch_batched(P, cps, s);
}

// Total number of residues (offsets[count]) for device or host offsets.
int batch_total(const uint64_t *offsets, uint32_t count, cudaStream_t s, uint64_t &total)
{
    cudaPointerAttributes attr;
    const cudaError_t e = cudaPointerGetAttributes(&attr, offsets + count);
    if (e != cudaSuccess) (void)cudaGetLastError();
    if (e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)) {
        FCIRC_CUDA_TRY(cudaMemcpyAsync(&total, offsets + count, 8, cudaMemcpyDeviceToHost, s));
        FCIRC_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        total = offsets[count];
    }
    return FCIRC_OK;
}

}  // namespace

struct BatchGraph {
    int dev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *scratch = nullptr;
};

}  // namespace fcirc

extern "C" {

int fcirc_matvec_batched(uint32_t p, const uint32_t *f, const uint64_t *offsets, const uint32_t *a,
                         const uint32_t *x, uint32_t *c, uint32_t count, void *stream)
{
    set_error("");
    if (!f || !offsets || !a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_batched: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (count == 0) return FCIRC_OK;
    uint64_t total = 0;
    FCIRC_TRY(batch_total(offsets, count, s, total));
    if (total > ((uint64_t)1 << 32)) return fail(FCIRC_EINVAL, "fcirc_matvec_batched: more than 2^32 residues");
    BatchParams P{};
    FCIRC_TRY(batch_setup(p, count, total, P));
    Arg af{f, (size_t)count * 4, true, false}, ao{offsets, ((size_t)count + 1) * 8, true, false};
    Arg aa{a, total * 4, true, false}, ax{x, total * 4, true, false}, ac{c, total * 4, false, true};
    Staging st;
    st.args = {&af, &ao, &aa, &ax, &ac};
    FCIRC_TRY(st.begin(s, batch_scratch_bytes(count, total)));
    P.f = static_cast<const uint32_t *>(af.d);
    P.offsets = static_cast<const uint64_t *>(ao.d);
    P.a = static_cast<const uint32_t *>(aa.d);
    P.x = static_cast<const uint32_t *>(ax.d);
    P.c = static_cast<uint32_t *>(ac.d);
    FCIRC_TRY(check_lt(P.a, total, p, s));
    FCIRC_TRY(check_lt(P.x, total, p, s));
    batch_carve(st.scratch, count, total, P);
    FCIRC_TRY(launch_with_config(P, tuned_config(p, count, total), s));
    return st.end();
}

int fcirc_batched_autotune(uint32_t p, const uint32_t *f, const uint64_t *offsets, const uint32_t *a,
                           const uint32_t *x, uint32_t *c, uint32_t count, void *stream, int *chosen)
{
    set_error("");
    if (!f || !offsets || !a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_batched_autotune: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (count == 0) return FCIRC_OK;
    uint64_t total = 0;
    FCIRC_TRY(batch_total(offsets, count, s, total));
    BatchParams P{};
    FCIRC_TRY(batch_setup(p, count, total, P));
    void *scratch = nullptr;
    FCIRC_TRY(scratch_acquire(s, batch_scratch_bytes(count, total), &scratch));
    P.f = f;
    P.offsets = offsets;
    P.a = a;
    P.x = x;
    P.c = c;
    batch_carve(scratch, count, total, P);
    cudaEvent_t e0, e1;
    FCIRC_CUDA_TRY(cudaEventCreate(&e0));
    FCIRC_CUDA_TRY(cudaEventCreate(&e1));
    int best = kDefaultBConfig;
    float best_ms = 1e30f;
    for (int cfg = 0; cfg < kNumBConfigs; ++cfg) {
        FCIRC_TRY(launch_with_config(P, cfg, s));   // warm-up
        float tot = 0.f;
        for (int r = 0; r < 3; ++r) {
            FCIRC_CUDA_TRY(cudaEventRecord(e0, s));
            FCIRC_TRY(launch_with_config(P, cfg, s));
            FCIRC_CUDA_TRY(cudaEventRecord(e1, s));
            FCIRC_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            FCIRC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (tot < best_ms) {
            best_ms = tot;
            best = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        g_tune[{dev, p, count, total}] = best;
        tune_store_locked();
    }
    if (chosen) *chosen = best;
    return FCIRC_OK;
}

int fcirc_batched_config(int index, int *ctas_per_sm, int *tile_log)
{
    if (index < 0 || index >= kNumBConfigs) return fail(FCIRC_EINVAL, "config index %d out of range", index);
    if (ctas_per_sm) *ctas_per_sm = kBConfigs[index].ctas_per_sm;
    if (tile_log) *tile_log = kBConfigs[index].big_log;
    return FCIRC_OK;
}

int fcirc_matvec_batched_graph(uint32_t p, const uint32_t *f, const uint64_t *offsets, const uint32_t *a,
                               const uint32_t *x, uint32_t *c, uint32_t count, uint64_t total_n, void *stream,
                               fcirc_graph_t *out)
{
    set_error("");
    if (!out || !f || !offsets || !a || !x || !c || count == 0)
        return fail(FCIRC_EINVAL, "fcirc_matvec_batched_graph: null pointer or empty batch");
    for (const void *ptr : {(const void *)f, (const void *)offsets, (const void *)a, (const void *)x, (const void *)c}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
            (void)cudaGetLastError();
            return fail(FCIRC_EINVAL, "fcirc_matvec_batched_graph: %p is not device memory", ptr);
        }
    }
    (void)stream;   // the graph is captured on a private stream (below)
    BatchParams P{};
    FCIRC_TRY(batch_setup(p, count, total_n, P));
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    BatchGraph *g = new BatchGraph();
    g->dev = dev;
    const size_t bytes = batch_scratch_bytes(count, total_n);
    if (dev_alloc(&g->scratch, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        delete g;
        return fail(FCIRC_ENOMEM, "fcirc_matvec_batched_graph: cudaMalloc(%zu)", bytes);
    }
    // every failure below releases the scratch and the handle
    auto give_up = [&](int status) {
        cudaFree(g->scratch);
        delete g;
        return status;
    };
    P.f = f;
    P.offsets = offsets;
    P.a = a;
    P.x = x;
    P.c = c;
    batch_carve(g->scratch, count, total_n, P);
    const int cfg = tuned_config(p, count, total_n);
    // capture on a private stream so that no other work lands in the graph
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return give_up(fail(FCIRC_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e)));
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaStreamDestroy(cs);
        return give_up(fail(FCIRC_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e)));
    }
    const int rc = launch_with_config(P, cfg, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc != FCIRC_OK || ce != cudaSuccess) {
        (void)cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return give_up(rc != FCIRC_OK ? rc : fail(FCIRC_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce)));
    }
    g->graph = graph;
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    if (ie != cudaSuccess) {
        (void)cudaGetLastError();
        cudaGraphDestroy(graph);
        return give_up(fail(FCIRC_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie)));
    }
    *out = reinterpret_cast<fcirc_graph_t>(g);
    return FCIRC_OK;
}

int fcirc_graph_launch(fcirc_graph_t graph, void *stream)
{
    set_error("");
    if (!graph) return fail(FCIRC_EINVAL, "fcirc_graph_launch: null graph");
    BatchGraph *g = reinterpret_cast<BatchGraph *>(graph);
    ProfScope ps("graph:batched", static_cast<cudaStream_t>(stream));
    FCIRC_CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return FCIRC_OK;
}

int fcirc_graph_destroy(fcirc_graph_t graph)
{
    set_error("");
    if (!graph) return FCIRC_OK;
    BatchGraph *g = reinterpret_cast<BatchGraph *>(graph);
    cudaSetDevice(g->dev);
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    cudaFree(g->scratch);
    delete g;
    return FCIRC_OK;
}

int fcirc_sync_status(void *stream)
{
    set_error("");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FCIRC_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t *w;
    FCIRC_TRY(device_status_word(&w));
    uint32_t v = 0;
    FCIRC_CUDA_TRY(cudaMemcpy(&v, w, 4, cudaMemcpyDeviceToHost));
    if (v) {
        FCIRC_CUDA_TRY(cudaMemset(w, 0, 4));
        if (v == FCIRC_EINVAL || v == FCIRC_ENOROOT)
            return fail((int)v, "a batched instance was invalid or had no root (device status %u)", v);
        return fail(FCIRC_ETIMEOUT, "a bounded device-side wait gave up (code %u)", v);
    }
    return FCIRC_OK;
}

int fcirc_set_checks(int on)
{
    set_error("");
    set_checks(on != 0);
    return FCIRC_OK;
}

int fcirc_debug_fail_alloc(int k)
{
    set_error("");
    debug_fail_alloc(k);
    return FCIRC_OK;
}

int fcirc_release(void)
{
    set_error("");
    release_scratch();
    release_plans();
    release_cplans();
    return FCIRC_OK;
}

}  // extern "C"
