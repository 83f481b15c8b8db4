// api.cu -- the C ABI (include/fcirc.h): argument checks, host/device
// staging, and the pass sequence of each entry point.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.hpp"
#include "kernels_mod.hpp"
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
    bool on_device;
    void *d;            // device pointer used by the kernels
};

int classify(Arg &a)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, a.user);
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
    }
    return FCIRC_OK;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Stages host arguments through the scratch pool; `extra` bytes of compute
// scratch follow the staging area.
struct Staging {
    std::vector<Arg *> args;
    cudaStream_t s;
    char *scratch = nullptr;
    bool any_host = false;

    int begin(cudaStream_t st, size_t extra)
    {
        s = st;
        size_t need = 0;
        for (Arg *a : args) {
            FCIRC_TRY(classify(*a));
            if (!a->on_device) {
                any_host = true;
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
                if (a->in && a->bytes)
                    FCIRC_CUDA_TRY(cudaMemcpyAsync(a->d, a->user, a->bytes, cudaMemcpyHostToDevice, s));
            }
        }
        scratch = cur;
        return FCIRC_OK;
    }

    int end()
    {
        if (!any_host) return FCIRC_OK;
        for (Arg *a : args)
            if (!a->on_device && a->out && a->bytes)
                FCIRC_CUDA_TRY(cudaMemcpyAsync(const_cast<void *>(a->user), a->d, a->bytes,
                                               cudaMemcpyDeviceToHost, s));
        FCIRC_CUDA_TRY(cudaStreamSynchronize(s));
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
    J.kt = pl->kt;
    J.store_lazy = lazy;
    return J;
}

}  // namespace

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
    const Src srcP{P, np, SRC_U16_REV}, srcQ{Q, nq, SRC_U16};
    const Plan &p0 = *pl[0];
    if (p0.k == 0) {
        TileParams tp;
        for (int q = 0; q < 3; ++q) tp.job[q] = tile_job(pl[q], srcP, srcQ, A[q], 0);
        tp.N = N;
        tp.logT = p0.logT;
        tp.D = p0.D;
        FCIRC_TRY(launch_tile(tp, 1, 3, s));
        return launch_crt_rot(A[0], A[1], A[2], N, out, nout, crt, s);
    }
    for (int i = 0; i < p0.npass; ++i) {
        StrFwdParams fp;
        for (int q = 0; q < 3; ++q) {
            Src sa = srcP, sx = srcQ;
            if (i > 0) {
                sa = Src{A[q], N, SRC_U32};
                sx = Src{X[q], N, SRC_U32};
            }
            fp.job[2 * q] = StrFwdJob{sa, A[q], pl[q]->d_ftw, kPrimes[q], 0};
            fp.job[2 * q + 1] = StrFwdJob{sx, X[q], pl[q]->d_ftw, kPrimes[q], 1};
        }
        fp.N = N;
        fp.logn = p0.m;
        fp.l0 = p0.pass_l0[i];
        fp.l1 = p0.pass_l1[i];
        fp.logW = 2;
        FCIRC_TRY(launch_strided_fwd(fp, 6, s));
    }
    {
        TileParams tp;
        for (int q = 0; q < 3; ++q)
            tp.job[q] = tile_job(pl[q], Src{A[q], N, SRC_U32}, Src{X[q], N, SRC_U32}, A[q], 1);
        tp.N = N;
        tp.logT = p0.logT;
        tp.D = p0.D;
        FCIRC_TRY(launch_tile(tp, (uint64_t)1 << p0.k, 3, s));
    }
    for (int i = p0.npass - 1; i >= 0; --i) {
        StrInvParams ip;
        for (int q = 0; q < 3; ++q) ip.job[q] = StrInvJob{A[q], A[q], pl[q]->d_fitw, kPrimes[q]};
        ip.nprime = 3;
        ip.N = N;
        ip.logn = p0.m;
        ip.l0 = p0.pass_l0[i];
        ip.l1 = p0.pass_l1[i];
        ip.logW = 2;
        ip.epi = (i == 0) ? EPI_CRT_ROT : EPI_LAZY;
        ip.dst64 = out;
        ip.nout = nout;
        ip.crt = crt;
        FCIRC_TRY(launch_strided_inv(ip, s));
    }
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
    if (!is_pow2(n)) return fail(FCIRC_EINVAL, "fcirc_matvec: n = %llu is not a power of two",
                                 (unsigned long long)n);
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
    if (pl->k == 0) {
        TileParams tp;
        tp.job[0] = tile_job(pl, Src{da, n, SRC_U32}, Src{dx, n, SRC_U32}, dc, 0);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        FCIRC_TRY(launch_tile(tp, 1, 1, s));
        return st.end();
    }
    uint32_t *xs = reinterpret_cast<uint32_t *>(st.scratch);
    for (int i = 0; i < pl->npass; ++i) {
        StrFwdParams fp;
        Src sa{da, n, SRC_U32}, sx{dx, n, SRC_U32};
        if (i > 0) {
            sa.ptr = dc;
            sx.ptr = xs;
        }
        fp.job[0] = StrFwdJob{sa, dc, pl->d_ftw, p, 0};
        fp.job[1] = StrFwdJob{sx, xs, pl->d_ftw, p, 1};
        fp.N = n;
        fp.logn = pl->m;
        fp.l0 = pl->pass_l0[i];
        fp.l1 = pl->pass_l1[i];
        fp.logW = 2;
        FCIRC_TRY(launch_strided_fwd(fp, 2, s));
    }
    {
        TileParams tp;
        tp.job[0] = tile_job(pl, Src{dc, n, SRC_U32}, Src{xs, n, SRC_U32}, dc, 1);
        tp.N = n;
        tp.logT = pl->logT;
        tp.D = pl->D;
        FCIRC_TRY(launch_tile(tp, (uint64_t)1 << pl->k, 1, s));
    }
    for (int i = pl->npass - 1; i >= 0; --i) {
        StrInvParams ip;
        ip.job[0] = StrInvJob{dc, dc, pl->d_fitw, p};
        ip.nprime = 1;
        ip.N = n;
        ip.logn = pl->m;
        ip.l0 = pl->pass_l0[i];
        ip.l1 = pl->pass_l1[i];
        ip.logW = 2;
        ip.epi = (i == 0) ? EPI_CANON : EPI_LAZY;
        ip.dst64 = nullptr;
        ip.nout = 0;
        FCIRC_TRY(launch_strided_inv(ip, s));
    }
    return st.end();
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
        return fail(FCIRC_ETIMEOUT, "a bounded device-side wait gave up (code %u)", v);
    }
    return FCIRC_OK;
}

int fcirc_release(void)
{
    set_error("");
    release_scratch();
    release_plans();
    return FCIRC_OK;
}

}  // extern "C"
