// plan.cu -- root chains and twiddle tables of the recursion (host side),
// cached per device, plus the scratch pool and status handling.
//
// For c = A x with A f-circulant of size n = 2^m (Section 2), the halving
// recursion visits node j of level l (block size n/2^l) with parameter
// f_{l,j} and splits it with s_{l,j} = sqrt(f_{l,j}) into children +s and -s
// (structure preservation, proof of Theorem 1).  The library fixes one
// consistent chain of square roots in closed form:
//
//   s_{l,j} = rho^(2^(L-l-1)) * psi_{2^(l+1)}^brv_l(j),  L = m - 1,
//
// rho a 2^L-th root of f, psi_m a primitive m-th root of unity taken from a
// fixed Omega (psi_m = Omega^(2^v/m)).  Squaring gives s_{l,j}^2 =
// (+/-) s_{l-1, j>>1} as required.  Inverse roots are the same products of
// rho^-1 and psi^-1 (Section 3.1 notes that inverse roots come from roots
// already computed).
//
// Inside a tile of 2^logT contiguous residues at depth k (node t of level k)
// the twiddle of relative level d, relative node j' factors as
//   s_{k+d, t 2^d + j'} = sigma_{t,d} * U[2^d + j'],
//   sigma_{t,d} = rho_t^(2^(D-1-d)),  rho_t = rho * psi_{2^L}^brv_k(t),
// with U the universal (f = 1) table of the prime; the kernels multiply the
// two on the fly, so only 2^k tile factors are stored instead of n twiddles.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/fcirc_plan.h"
#include "common.hpp"
#include "kernels_mod.hpp"
#include "gfp2.hpp"
#include "ring.hpp"

namespace fcirc {

// ---------------------------------------------------------------------------
// error detail

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return status;
}

const char *last_error_detail() { return g_err; }

// ---------------------------------------------------------------------------
// scratch pool: one growing buffer per (device, stream)

namespace {
struct ScratchBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, cudaStream_t>, ScratchBuf> g_scratch;
std::map<int, uint32_t *> g_status;
}  // namespace

namespace {
std::atomic<int> g_fail_alloc{-1};
}

void debug_fail_alloc(int k) { g_fail_alloc.store(k < 0 ? -1 : k); }

cudaError_t dev_alloc(void **ptr, size_t bytes)
{
    int k = g_fail_alloc.load();
    while (k >= 0) {
        if (g_fail_alloc.compare_exchange_weak(k, k - 1)) {
            if (k == 0) {
                *ptr = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(ptr, bytes);
}

int scratch_acquire(cudaStream_t s, size_t bytes, void **out)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchBuf &b = g_scratch[{dev, s}];
    if (b.bytes < bytes) {
        if (b.ptr) {
            FCIRC_CUDA_TRY(cudaDeviceSynchronize());
            FCIRC_CUDA_TRY(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + (bytes >> 3);
        want = (want + 0xFFFFF) & ~(size_t)0xFFFFF;
        cudaError_t e = dev_alloc(&b.ptr, want);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b.ptr = nullptr;
            return fail(FCIRC_ENOMEM, "scratch: cudaMalloc(%zu) failed: %s", want,
                        cudaGetErrorString(e));
        }
        b.bytes = want;
    }
    *out = b.ptr;
    return FCIRC_OK;
}

int device_status_word(uint32_t **out)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    uint32_t *&w = g_status[dev];
    if (!w) {
        // through dev_alloc, so that the allocation fault injection reaches it
        void *ptr = nullptr;
        const cudaError_t e = dev_alloc(&ptr, 256);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FCIRC_ENOMEM, "status word: cudaMalloc(256) failed: %s", cudaGetErrorString(e));
        }
        const cudaError_t z = cudaMemset(ptr, 0, 256);
        if (z != cudaSuccess) {
            (void)cudaFree(ptr);
            return fail(FCIRC_ECUDA, "status word: cudaMemset failed: %s", cudaGetErrorString(z));
        }
        w = static_cast<uint32_t *>(ptr);
    }
    *out = w;
    return FCIRC_OK;
}

void release_scratch()
{
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    for (auto &kv : g_scratch)
        if (kv.second.ptr) {
            cudaSetDevice(kv.first.first);
            cudaDeviceSynchronize();
            cudaFree(kv.second.ptr);
        }
    g_scratch.clear();
    // the status words stay: they are tiny and their address may be cached
    // by callers of fcirc_sync_status in flight
}

// ---------------------------------------------------------------------------
// per-prime universal tables

namespace {
std::mutex g_plan_mu;
std::map<std::pair<int, uint32_t>, PrimeTables *> g_primes;
std::map<std::tuple<int, uint32_t, uint32_t, uint64_t>, Plan *> g_plans;
}  // namespace

using namespace host;

static int upload(void **dptr, const void *src, size_t bytes)
{
    if (bytes == 0) {
        *dptr = nullptr;
        return FCIRC_OK;
    }
    cudaError_t e = dev_alloc(dptr, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *dptr = nullptr;
        return fail(FCIRC_ENOMEM, "plan: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    e = cudaMemcpy(*dptr, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(*dptr);
        *dptr = nullptr;
        return fail(FCIRC_ECUDA, "plan: cudaMemcpy(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return FCIRC_OK;
}

static bool prime_ok(uint32_t p) { return p >= 3 && p < (1u << 30) && is_prime(p); }

// U[2^d + j] = psi_{2^(d+1)}^brv_d(j) for d < min(kUnivLog, v); inverse in Ui.
static void universal_tables(uint32_t p, uint32_t Om, int v, std::vector<uint32_t> &U,
                             std::vector<uint32_t> &Ui)
{
    U.assign((size_t)1 << kUnivLog, 0);
    Ui.assign((size_t)1 << kUnivLog, 0);
    for (int d = 0; d < kUnivLog && d + 1 <= v; ++d) {
        uint32_t psi = powmod(Om, (uint64_t)1 << (v - d - 1), p);  // primitive 2^(d+1)-th
        uint32_t psii = invmod(psi, p);
        uint64_t cnt = (uint64_t)1 << d;
        std::vector<uint32_t> pw(cnt), pwi(cnt);
        uint32_t c = 1, ci = 1;
        for (uint64_t i = 0; i < cnt; ++i) {
            pw[i] = c;
            pwi[i] = ci;
            c = mulmod(c, psi, p);
            ci = mulmod(ci, psii, p);
        }
        for (uint64_t j = 0; j < cnt; ++j) {
            U[cnt + j] = pw[bitrev(j, d)];
            Ui[cnt + j] = pwi[bitrev(j, d)];
        }
    }
}

int prime_tables(uint32_t p, const PrimeTables **out)
{
    if (!prime_ok(p)) return fail(FCIRC_EINVAL, "p = %u is not an odd prime below 2^30", p);
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_primes.find({dev, p});
    if (it != g_primes.end()) {
        *out = it->second;
        return FCIRC_OK;
    }
    PrimeTables *t = new PrimeTables();
    t->p = p;
    t->v = two_adic(p);
    t->omega = omega(p);
    // p^-1 mod 2^32 by Newton iteration (p odd)
    uint32_t inv = p;
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    t->pinv = inv;
    std::vector<uint32_t> U, Ui;
    universal_tables(p, t->omega, t->v, U, Ui);
    int s = upload((void **)&t->d_U, U.data(), U.size() * 4);
    if (s == FCIRC_OK) s = upload((void **)&t->d_Ui, Ui.data(), Ui.size() * 4);
    if (s != FCIRC_OK) {
        cudaFree(t->d_U);
        cudaFree(t->d_Ui);
        delete t;
        return s;
    }
    g_primes[{dev, p}] = t;
    *out = t;
    return FCIRC_OK;
}

static Tw make_tw(uint32_t w, uint32_t p)
{
    Tw t;
    t.w = w % p;
    t.wp = shoup_quot(t.w, p);
    return t;
}

// Plan numbers that do not depend on the device.
struct PlanShape {
    int m, L, k, logT, D;
    uint32_t rho;
};

static int plan_shape(uint32_t p, uint32_t f, uint64_t n, PlanShape &sh)
{
    if (!prime_ok(p)) return fail(FCIRC_EINVAL, "p = %u is not an odd prime below 2^30", p);
    if (!is_pow2(n)) return fail(FCIRC_EINVAL, "n = %llu is not a power of two", (unsigned long long)n);
    sh.m = ilog2(n);
    if (sh.m > kMaxLogN) return fail(FCIRC_EINVAL, "n = 2^%d exceeds 2^%d", sh.m, kMaxLogN);
    if (sh.m < 1) return fail(FCIRC_EINVAL, "n = 1 has no plan");
    sh.L = sh.m - 1;
    int v = two_adic(p);
    if (sh.L > v)
        return fail(FCIRC_ENOROOT, "n = 2^%d needs a primitive 2^%d-th root of unity; p - 1 has only 2^%d",
                    sh.m, sh.L, v);
    if (f % p == 0) return fail(FCIRC_ENOROOT, "f = 0 has no inverse (Theorem 1)");
    if (!nth_root_2k(f, sh.L, p, sh.rho))
        return fail(FCIRC_ENOROOT, "f = %u has no 2^%d-th root mod %u (Theorem 1)", f, sh.L, p);
    if (sh.m <= kTileLogMax) {
        sh.k = 0;
        sh.logT = sh.m;
    } else {
        sh.logT = kTileLogMax;
        sh.k = sh.m - kTileLogMax;
    }
    sh.D = sh.logT - 1;
    return FCIRC_OK;
}

int plan_node_twiddle_host(uint32_t p, uint32_t f, uint64_t n, int level, uint64_t j,
                           uint32_t *s, uint32_t *si)
{
    PlanShape sh;
    FCIRC_TRY(plan_shape(p, f, n, sh));
    if (level < 0 || level >= sh.L || j >= ((uint64_t)1 << level))
        return fail(FCIRC_EINVAL, "node (%d, %llu) outside the %d halving levels", level,
                    (unsigned long long)j, sh.L);
    int v = two_adic(p);
    uint32_t Om = omega(p);
    uint32_t P = powmod(sh.rho, (uint64_t)1 << (sh.L - level - 1), p);
    uint32_t psi = powmod(Om, (uint64_t)1 << (v - level - 1), p);
    uint32_t w = mulmod(P, powmod(psi, bitrev(j, level), p), p);
    *s = w;
    *si = invmod(w, p);
    return FCIRC_OK;
}

static int build_plan(uint32_t p, uint32_t f, uint64_t n, Plan *pl)
{
    PlanShape sh;
    FCIRC_TRY(plan_shape(p, f, n, sh));
    const PrimeTables *pt;
    FCIRC_TRY(prime_tables(p, &pt));
    pl->p = p;
    pl->f = f % p;
    pl->n = n;
    pl->m = sh.m;
    pl->L = sh.L;
    pl->k = sh.k;
    pl->logT = sh.logT;
    pl->D = sh.D;
    pl->rho = sh.rho;
    pl->pt = pt;
    // strided passes over [0, k), at most kPassLogMax levels each, balanced
    pl->npass = (sh.k + kPassLogMax - 1) / kPassLogMax;
    for (int i = 0, l = 0; i < pl->npass; ++i) {
        int take = (sh.k - l) / (pl->npass - i);
        pl->pass_l0[i] = l;
        pl->pass_l1[i] = l + take;
        l += take;
    }
    // leaf scale 2^32 * 2^-L mod p
    uint32_t two32 = (uint32_t)(((uint64_t)1 << 32) % p);
    uint32_t inv2L = powmod(invmod(2, p), sh.L, p);
    pl->kt = make_tw(mulmod(two32, inv2L, p), p);

    const uint32_t Om = pt->omega;
    const int v = pt->v;
    const uint32_t rho = sh.rho, rhoi = invmod(sh.rho, p);
    // ---- top-level twiddles s_{l,j}, l < k (heap order)
    if (sh.k > 0) {
        size_t cnt = (size_t)1 << sh.k;
        std::vector<Tw> ftw(cnt), fitw(cnt);
        ftw[0] = fitw[0] = Tw{0, 0};
        for (int l = 0; l < sh.k; ++l) {
            uint32_t P = powmod(rho, (uint64_t)1 << (sh.L - l - 1), p);
            uint32_t Pi = powmod(rhoi, (uint64_t)1 << (sh.L - l - 1), p);
            uint32_t psi = powmod(Om, (uint64_t)1 << (v - l - 1), p);
            uint32_t psii = invmod(psi, p);
            uint64_t nn = (uint64_t)1 << l;
            std::vector<uint32_t> pw(nn), pwi(nn);
            uint32_t c = 1, ci = 1;
            for (uint64_t i = 0; i < nn; ++i) {
                pw[i] = c;
                pwi[i] = ci;
                c = mulmod(c, psi, p);
                ci = mulmod(ci, psii, p);
            }
            for (uint64_t j = 0; j < nn; ++j) {
                ftw[nn + j] = make_tw(mulmod(P, pw[bitrev(j, l)], p), p);
                fitw[nn + j] = make_tw(mulmod(Pi, pwi[bitrev(j, l)], p), p);
            }
        }
        FCIRC_TRY(upload((void **)&pl->d_ftw, ftw.data(), cnt * sizeof(Tw)));
        FCIRC_TRY(upload((void **)&pl->d_fitw, fitw.data(), cnt * sizeof(Tw)));
        // group-ordered copies for the register-staged column passes: stage s
        // of a pass over levels [l0, l1), group block gb (a node of level
        // l0 + d0(s)), local level d, node j -> slot 16 gb + 16 - 2^(d+1) + j
        std::vector<Tw> g, gi;
        for (int i = 0; i < pl->npass; ++i) {
            const int l0 = pl->pass_l0[i], lf = pl->pass_l1[i] - l0;
            pl->pass_goff[i] = (int)g.size();
            int off = 0;
            for (int st = 0; st < col_nstage(lf); ++st) {
                pl->stage_off[i][st] = off;
                const int d0 = col_d0(lf, st), nl = col_nl(lf, st);
                const uint64_t ngb = (uint64_t)1 << (l0 + d0);
                g.resize(g.size() + ngb * 16, Tw{0, 0});
                gi.resize(gi.size() + ngb * 16, Tw{0, 0});
                Tw *G = g.data() + pl->pass_goff[i] + off, *GI = gi.data() + pl->pass_goff[i] + off;
                for (uint64_t gb = 0; gb < ngb; ++gb)
                    for (int d = 0; d < nl; ++d)
                        for (uint64_t j = 0; j < ((uint64_t)1 << d); ++j) {
                            const uint64_t heap = ((uint64_t)1 << (l0 + d0 + d)) + (gb << d) + j;
                            G[gb * 16 + 16 - (2 << d) + j] = ftw[heap];
                            GI[gb * 16 + 16 - (2 << d) + j] = fitw[heap];
                        }
                off += (int)(ngb * 16);
            }
        }
        FCIRC_TRY(upload((void **)&pl->d_gtw, g.data(), g.size() * sizeof(Tw)));
        FCIRC_TRY(upload((void **)&pl->d_gitw, gi.data(), gi.size() * sizeof(Tw)));
        // the last stage of each pass, ordered by slot pair
        std::vector<Tw> gl, gil;
        for (int i = 0; i < pl->npass; ++i) {
            const int l0 = pl->pass_l0[i], lf = pl->pass_l1[i] - l0, st = col_nstage(lf) - 1;
            const uint64_t ngb = (uint64_t)1 << (l0 + col_d0(lf, st));
            pl->pass_loff[i] = (int)gl.size();
            gl.resize(gl.size() + ngb * 16, Tw{0, 0});
            gil.resize(gil.size() + ngb * 16, Tw{0, 0});
            const Tw *G = g.data() + pl->pass_goff[i] + pl->stage_off[i][st];
            const Tw *GI = gi.data() + pl->pass_goff[i] + pl->stage_off[i][st];
            for (uint64_t gb = 0; gb < ngb; ++gb)
                for (int slot = 0; slot < 16; ++slot) {
                    const uint64_t e = 2 * ((uint64_t)(slot >> 1) * ngb + gb) + (slot & 1);
                    gl[pl->pass_loff[i] + e] = G[gb * 16 + slot];
                    gil[pl->pass_loff[i] + e] = GI[gb * 16 + slot];
                }
        }
        FCIRC_TRY(upload((void **)&pl->d_gtwl, gl.data(), gl.size() * sizeof(Tw)));
        FCIRC_TRY(upload((void **)&pl->d_gitwl, gil.data(), gil.size() * sizeof(Tw)));
    }
    // ---- tile factors: rho_t = rho * Psi^brv_k(t), sigma_{t,d} = rho_t^(2^(D-1-d))
    {
        size_t ntile = (size_t)1 << sh.k;
        std::vector<uint32_t> sig(ntile * (size_t)(sh.D > 0 ? sh.D : 1) * 6, 0);
        std::vector<Tw> trho(ntile);
        uint32_t Psi = powmod(Om, (uint64_t)1 << (v - sh.L), p);   // primitive 2^L-th
        uint32_t Psii = invmod(Psi, p);
        std::vector<uint32_t> pw(ntile), pwi(ntile);
        uint32_t c = 1, ci = 1;
        for (size_t i = 0; i < ntile; ++i) {
            pw[i] = c;
            pwi[i] = ci;
            c = mulmod(c, Psi, p);
            ci = mulmod(ci, Psii, p);
        }
        for (size_t t = 0; t < ntile; ++t) {
            uint32_t b = sh.k ? bitrev(t, sh.k) : 0;
            uint32_t rt = mulmod(rho, pw[b], p), rti = mulmod(rhoi, pwi[b], p);
            trho[t] = make_tw(rt, p);
            uint32_t sgm = rt, sgmi = rti;
            for (int d = sh.D - 1; d >= 0; --d) {
                uint32_t *e = &sig[(t * sh.D + d) * 6];
                e[0] = sgm;
                shoup_quot64(sgm, p, e[1], e[2]);
                e[3] = sgmi;
                shoup_quot64(sgmi, p, e[4], e[5]);
                sgm = mulmod(sgm, sgm, p);
                sgmi = mulmod(sgmi, sgmi, p);
            }
        }
        FCIRC_TRY(upload((void **)&pl->d_sig, sig.data(), sig.size() * 4));
        FCIRC_TRY(upload((void **)&pl->d_rho, trho.data(), trho.size() * sizeof(Tw)));
    }
    return FCIRC_OK;
}

static void free_plan_tables(Plan *pl)
{
    cudaFree(pl->d_ftw);
    cudaFree(pl->d_fitw);
    cudaFree(pl->d_sig);
    cudaFree(pl->d_rho);
    cudaFree(pl->d_gtw);
    cudaFree(pl->d_gitw);
    cudaFree(pl->d_gtwl);
    cudaFree(pl->d_gitwl);
}

int get_plan(uint32_t p, uint32_t f, uint64_t n, const Plan **out)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find({dev, p, f % (p ? p : 1), n});
        if (it != g_plans.end()) {
            *out = it->second;
            return FCIRC_OK;
        }
    }
    Plan *pl = new Plan();
    int s = build_plan(p, f, n, pl);
    if (s != FCIRC_OK) {
        free_plan_tables(pl);
        delete pl;
        return s;
    }
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto key = std::make_tuple(dev, p, f % p, n);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {  // built concurrently by another thread
        free_plan_tables(pl);
        delete pl;
        *out = it->second;
        return FCIRC_OK;
    }
    g_plans[key] = pl;
    *out = pl;
    return FCIRC_OK;
}

void release_plans()
{
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto &kv : g_plans) {
        cudaSetDevice(std::get<0>(kv.first));
        cudaDeviceSynchronize();
        Plan *pl = kv.second;
        free_plan_tables(pl);
        delete pl;
    }
    g_plans.clear();
    for (auto &kv : g_primes) {
        cudaSetDevice(kv.first.first);
        cudaFree(kv.second->d_U);
        cudaFree(kv.second->d_Ui);
        delete kv.second;
    }
    g_primes.clear();
}

}  // namespace fcirc

// ---------------------------------------------------------------------------
// fcirc_plan.h

extern "C" {

int fcirc_nth_root(uint32_t p, uint32_t f, uint32_t log2k, uint32_t *root)
{
    using namespace fcirc;
    if (!root) return fail(FCIRC_EINVAL, "null output");
    if (!prime_ok(p)) return fail(FCIRC_EINVAL, "p = %u is not an odd prime below 2^30", p);
    if (log2k > 40) return fail(FCIRC_EINVAL, "log2k = %u too large", log2k);
    uint32_t r;
    if (!host::nth_root_2k(f, (int)log2k, p, r))
        return fail(FCIRC_ENOROOT, "f = %u has no 2^%u-th root mod %u", f, log2k, p);
    *root = r;
    return FCIRC_OK;
}

int fcirc_gf_nth_root(uint32_t f_re, uint32_t f_im, uint32_t log2k, uint32_t *r_re, uint32_t *r_im)
{
    using namespace fcirc;
    if (!r_re || !r_im) return fail(FCIRC_EINVAL, "null output");
    if (f_re >= gf::P || f_im >= gf::P) return fail(FCIRC_EINVAL, "f not canonical mod 2^31 - 1");
    if (log2k > 30) return fail(FCIRC_EINVAL, "log2k = %u too large", log2k);
    gf::E r;
    if (!gf::root_2k(gf::E{f_re, f_im}, (int)log2k, r))
        return fail(FCIRC_ENOROOT, "%u + %u sqrt 3 has no 2^%u-th root", f_re, f_im, log2k);
    *r_re = r.re;
    *r_im = r.im;
    return FCIRC_OK;
}

int fcirc_node_twiddle(uint32_t p, uint32_t f, uint64_t n, uint32_t level, uint64_t j,
                       uint32_t *s, uint32_t *s_inv)
{
    if (!s || !s_inv) return fcirc::fail(FCIRC_EINVAL, "null output");
    return fcirc::plan_node_twiddle_host(p, f, n, (int)level, j, s, s_inv);
}

int fcirc_leaf_param(uint32_t p, uint32_t f, uint64_t n, uint64_t j, uint32_t *phi)
{
    using namespace fcirc;
    if (!phi) return fail(FCIRC_EINVAL, "null output");
    if (n == 2) {
        PlanShape sh;
        FCIRC_TRY(plan_shape(p, f, n, sh));
        if (j != 0) return fail(FCIRC_EINVAL, "leaf %llu out of range", (unsigned long long)j);
        *phi = f % p;
        return FCIRC_OK;
    }
    if (!is_pow2(n) || n < 2 || j >= n / 2)
        return fail(FCIRC_EINVAL, "leaf %llu out of range", (unsigned long long)j);
    int L = ilog2(n) - 1;
    uint32_t s, si;
    FCIRC_TRY(plan_node_twiddle_host(p, f, n, L - 1, j >> 1, &s, &si));
    *phi = (j & 1) ? (p - s) % p : s;
    return FCIRC_OK;
}

int fcirc_twiddle_from_factor(uint32_t p, uint32_t u, uint32_t sigma, uint32_t *w,
                              uint32_t *w_shoup)
{
    using namespace fcirc;
    if (!w || !w_shoup) return fail(FCIRC_EINVAL, "null output");
    if (!prime_ok(p) || u >= p || sigma >= p)
        return fail(FCIRC_EINVAL, "need prime p < 2^30 and u, sigma < p");
    uint32_t hi, lo;
    host::shoup_quot64(sigma, p, hi, lo);
    Tw t = twiddle_from(u, sigma, hi, lo, p);
    *w = t.w;
    *w_shoup = t.wp;
    return FCIRC_OK;
}

}  // extern "C"
