// noalloc.cu -- fcirc_matvec_noalloc: the modular f-circulant product for
// callers that must not have the library allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: code that runs with a
// fixed memory budget reserved up front (an inference server that carved
// the GPU into pools at start-up, a process whose allocator must stay
// deterministic), or code that must never trigger the implicit device-wide
// synchronisation a cudaMalloc/cudaFree can cause in the middle of its
// streams.  fcirc_matvec keeps scratch and plan tables in memory it
// allocates on first use; this entry point instead keeps both in one
// file-scope device array that exists from the moment the library is
// loaded, so a call never allocates.
//
// Layout of the array (kNoallocBytes in total):
//   [0, kScratchBytes)          the vector side's intermediate (n residues)
//   [kScratchBytes, ...)        this call's plan tables: universal roots of
//                               unity, top-level twiddles (heap and group
//                               order), tile factors and tile roots.
//
// The tables are written by the host before the kernels are enqueued (a
// plain host-to-device copy into the array), and every scratch word a
// kernel reads was written earlier by the same call, so nothing has to be
// cleared between calls.
#include <mutex>
#include <vector>

#include "../../include/fcirc.h"
#include "common.hpp"
#include "kernels_mod.hpp"
#include "ring.hpp"

namespace fcirc {
namespace {
constexpr int kNoallocMaxLog = 20;                                   // n <= 2^20
constexpr size_t kScratchBytes = (size_t)4 << kNoallocMaxLog;        // 4 MiB
constexpr size_t kTableBytes = (size_t)1 << 20;                      // 1 MiB
constexpr size_t kNoallocBytes = kScratchBytes + kTableBytes;        // 5 MiB
}  // namespace
}  // namespace fcirc

// The whole working area of fcirc_matvec_noalloc.  Every GPU that loads the
// library holds these 5 MiB until the process exits.
static __device__ __align__(256) unsigned char g_fcirc_noalloc_area[fcirc::kNoallocBytes];

namespace fcirc {
namespace {

// Host copy of one plan, laid out for the array.
struct HostPlan {
    int m, L, k, logT, D;
    int npass, l0[4], l1[4], stage_off[4][3], goff[4];
    uint32_t pinv;
    Tw kt;
    std::vector<uint32_t> U, Ui, sig;
    std::vector<Tw> ftw, fitw, g, gi, gl, gil, rho;
};

Tw tw_of(uint32_t w, uint32_t p)
{
    Tw t;
    t.w = w % p;
    t.wp = host::shoup_quot(t.w, p);
    return t;
}

int build_host_plan(uint32_t p, uint32_t f, uint64_t n, HostPlan &h)
{
    using namespace host;
    if (p < 3 || p >= (1u << 30) || !is_prime(p)) return fail(FCIRC_EINVAL, "p = %u is not an odd prime below 2^30", p);
    h.m = ilog2(n);
    h.L = h.m - 1;
    const int v = two_adic(p);
    if (h.L > v) return fail(FCIRC_ENOROOT, "n = 2^%d needs a primitive 2^%d-th root of unity mod %u", h.m, h.L, p);
    if (f % p == 0) return fail(FCIRC_ENOROOT, "f = 0 has no inverse (Theorem 1)");
    uint32_t rho;
    if (!nth_root_2k(f, h.L, p, rho)) return fail(FCIRC_ENOROOT, "f = %u has no 2^%d-th root mod %u", f, h.L, p);
    const uint32_t rhoi = invmod(rho, p);
    const uint32_t Om = omega(p);
    if (h.m <= kTileLogMax) {
        h.k = 0;
        h.logT = h.m;
    } else {
        h.logT = kTileLogMax;
        h.k = h.m - kTileLogMax;
    }
    h.D = h.logT - 1;
    h.npass = h.k > 0 ? 1 : 0;   // k <= 8 here: one strided pass
    h.l0[0] = 0;
    h.l1[0] = h.k;
    uint32_t inv = p;
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    h.pinv = inv;
    h.kt = tw_of(mulmod((uint32_t)(((uint64_t)1 << 32) % p), powmod(invmod(2, p), h.L, p), p), p);
    // universal tables U[2^d + j] = psi_{2^(d+1)}^brv_d(j)
    h.U.assign((size_t)1 << kUnivLog, 0);
    h.Ui.assign((size_t)1 << kUnivLog, 0);
    for (int d = 0; d < kUnivLog && d + 1 <= v; ++d) {
        const uint32_t psi = powmod(Om, (uint64_t)1 << (v - d - 1), p), psii = invmod(psi, p);
        const uint64_t cnt = (uint64_t)1 << d;
        uint32_t c = 1, ci = 1;
        for (uint64_t i = 0; i < cnt; ++i) {   // psi^i lands at position brv_d(i)
            h.U[cnt + bitrev(i, d)] = c;
            h.Ui[cnt + bitrev(i, d)] = ci;
            c = mulmod(c, psi, p);
            ci = mulmod(ci, psii, p);
        }
    }
    // top-level twiddles s_{l,j}, l < k, heap order, then in group order
    if (h.k > 0) {
        const size_t cnt = (size_t)1 << h.k;
        h.ftw.assign(cnt, Tw{0, 0});
        h.fitw.assign(cnt, Tw{0, 0});
        for (int l = 0; l < h.k; ++l) {
            const uint32_t P = powmod(rho, (uint64_t)1 << (h.L - l - 1), p);
            const uint32_t Pi = powmod(rhoi, (uint64_t)1 << (h.L - l - 1), p);
            const uint32_t psi = powmod(Om, (uint64_t)1 << (v - l - 1), p), psii = invmod(psi, p);
            uint32_t c = 1, ci = 1;
            for (uint64_t i = 0; i < ((uint64_t)1 << l); ++i) {
                h.ftw[((size_t)1 << l) + bitrev(i, l)] = tw_of(mulmod(P, c, p), p);
                h.fitw[((size_t)1 << l) + bitrev(i, l)] = tw_of(mulmod(Pi, ci, p), p);
                c = mulmod(c, psi, p);
                ci = mulmod(ci, psii, p);
            }
        }
        const int lf = h.k;
        h.goff[0] = 0;
        int off = 0;
        for (int st = 0; st < col_nstage(lf); ++st) {
            h.stage_off[0][st] = off;
            const int d0 = col_d0(lf, st), nl = col_nl(lf, st);
            const uint64_t ngb = (uint64_t)1 << d0;
            h.g.resize(off + ngb * 16, Tw{0, 0});
            h.gi.resize(off + ngb * 16, Tw{0, 0});
            for (uint64_t gb = 0; gb < ngb; ++gb)
                for (int d = 0; d < nl; ++d)
                    for (uint64_t j = 0; j < ((uint64_t)1 << d); ++j) {
                        const uint64_t heap = ((uint64_t)1 << (d0 + d)) + (gb << d) + j;
                        h.g[off + gb * 16 + 16 - (2 << d) + j] = h.ftw[heap];
                        h.gi[off + gb * 16 + 16 - (2 << d) + j] = h.fitw[heap];
                    }
            off += (int)(ngb * 16);
        }
        // the last stage again, ordered by slot pair (ColFwdJob::gtwl)
        const int st = col_nstage(lf) - 1;
        const uint64_t ngb = (uint64_t)1 << col_d0(lf, st);
        h.gl.assign(ngb * 16, Tw{0, 0});
        h.gil.assign(ngb * 16, Tw{0, 0});
        for (uint64_t gb = 0; gb < ngb; ++gb)
            for (int slot = 0; slot < 16; ++slot) {
                const uint64_t e = 2 * ((uint64_t)(slot >> 1) * ngb + gb) + (slot & 1);
                h.gl[e] = h.g[h.stage_off[0][st] + gb * 16 + slot];
                h.gil[e] = h.gi[h.stage_off[0][st] + gb * 16 + slot];
            }
    }
    // tile factors sigma_{t,d} = rho_t^(2^(D-1-d)), rho_t = rho psi_{2^L}^brv_k(t)
    const size_t ntile = (size_t)1 << h.k;
    h.sig.assign(ntile * (size_t)(h.D > 0 ? h.D : 1) * 6, 0);
    h.rho.assign(ntile, Tw{0, 0});
    const uint32_t Psi = powmod(Om, (uint64_t)1 << (v - h.L), p), Psii = invmod(Psi, p);
    for (size_t t = 0; t < ntile; ++t) {
        const uint32_t b = h.k ? bitrev(t, h.k) : 0;
        uint32_t sg = mulmod(rho, powmod(Psi, b, p), p), sgi = mulmod(rhoi, powmod(Psii, b, p), p);
        h.rho[t] = tw_of(sg, p);
        for (int d = h.D - 1; d >= 0; --d) {
            uint32_t *e = &h.sig[(t * h.D + d) * 6];
            e[0] = sg;
            shoup_quot64(sg, p, e[1], e[2]);
            e[3] = sgi;
            shoup_quot64(sgi, p, e[4], e[5]);
            sg = mulmod(sg, sg, p);
            sgi = mulmod(sgi, sgi, p);
        }
    }
    return FCIRC_OK;
}

// Device pointers of the tables inside the array.
struct DevTables {
    uint32_t *U, *Ui, *sig;
    Tw *ftw, *fitw, *g, *gi, *gl, *gil, *rho;
};

// Per-device state: the array's device address (looked up once per device)
// and the (p, f, n) whose tables the array currently holds.
struct DevState {
    bool ready = false;
    unsigned char *base = nullptr;
    bool tables_valid = false;      // the array holds the tables of (p, f, n)
    uint32_t p = 0, f = 0;
    uint64_t n = 0;
    HostPlan h;                     // scalars of that plan (vectors released)
    DevTables t;
};
std::mutex g_mu;
DevState g_dev[64];

// Carves the table area of the array and copies the host plan into it.
int upload_tables(unsigned char *base, const HostPlan &h, DevTables &t, cudaStream_t s)
{
    size_t off = kScratchBytes;
    auto carve = [&](size_t bytes) {
        unsigned char *ptr = base + off;
        off += (bytes + 255) & ~(size_t)255;
        return ptr;
    };
    t.U = reinterpret_cast<uint32_t *>(carve(h.U.size() * 4));
    t.Ui = reinterpret_cast<uint32_t *>(carve(h.Ui.size() * 4));
    t.sig = reinterpret_cast<uint32_t *>(carve(h.sig.size() * 4));
    t.rho = reinterpret_cast<Tw *>(carve(h.rho.size() * sizeof(Tw)));
    t.ftw = reinterpret_cast<Tw *>(carve(h.ftw.size() * sizeof(Tw)));
    t.fitw = reinterpret_cast<Tw *>(carve(h.fitw.size() * sizeof(Tw)));
    t.g = reinterpret_cast<Tw *>(carve(h.g.size() * sizeof(Tw)));
    t.gi = reinterpret_cast<Tw *>(carve(h.gi.size() * sizeof(Tw)));
    t.gl = reinterpret_cast<Tw *>(carve(h.gl.size() * sizeof(Tw)));
    t.gil = reinterpret_cast<Tw *>(carve(h.gil.size() * sizeof(Tw)));
    if (off > kNoallocBytes)
        return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: plan tables exceed the static area");
    auto put = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes) FCIRC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return FCIRC_OK;
    };
    FCIRC_TRY(put(t.U, h.U.data(), h.U.size() * 4));
    FCIRC_TRY(put(t.Ui, h.Ui.data(), h.Ui.size() * 4));
    FCIRC_TRY(put(t.sig, h.sig.data(), h.sig.size() * 4));
    FCIRC_TRY(put(t.rho, h.rho.data(), h.rho.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.ftw, h.ftw.data(), h.ftw.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.fitw, h.fitw.data(), h.fitw.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.g, h.g.data(), h.g.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.gi, h.gi.data(), h.gi.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.gl, h.gl.data(), h.gl.size() * sizeof(Tw)));
    FCIRC_TRY(put(t.gil, h.gil.data(), h.gil.size() * sizeof(Tw)));
    // copies from pageable memory have consumed their source when they return
    return FCIRC_OK;
}

int is_device_ptr(const void *ptr, int dev, bool &ok)
{
    cudaPointerAttributes attr;
    const cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ok = false;
        return FCIRC_OK;
    }
    ok = (attr.type == cudaMemoryTypeDevice && attr.device == dev) || attr.type == cudaMemoryTypeManaged;
    return FCIRC_OK;
}

}  // namespace
}  // namespace fcirc

using namespace fcirc;

extern "C" int fcirc_matvec_noalloc(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x,
                                    uint32_t *c, uint64_t n, void *stream)
{
    set_error("");
    if (!a || !x || !c) return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: null pointer");
    if (!is_pow2(n) || n < 2)
        return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: n = %llu must be a power of two >= 2",
                    (unsigned long long)n);
    if (n > ((uint64_t)1 << kNoallocMaxLog))
        return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: n = %llu exceeds the static limit 2^%d (use fcirc_matvec)",
                    (unsigned long long)n, kNoallocMaxLog);
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: device %d out of range", dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The table cache below is host state: a call recorded into a graph could
    // not know which tables the array holds when the graph is replayed, and
    // a table upload recorded from a host vector freed on return would copy
    // garbage.  So a call on a stream that is being captured does nothing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCIRC_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: the stream is being captured into a graph");

    for (const void *ptr : {(const void *)a, (const void *)x, (const void *)c}) {
        bool ok;
        FCIRC_TRY(is_device_ptr(ptr, dev, ok));
        if (!ok) return fail(FCIRC_EINVAL, "fcirc_matvec_noalloc: %p is not device memory of device %d", ptr, dev);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &ds = g_dev[dev];
    if (!ds.ready) {
        // set-up, once per device, with that device current: the array's name
        // is only a host-side stand-in, the kernels need its device address
        void *ptr = nullptr;
        FCIRC_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_fcirc_noalloc_area));
        ds.base = static_cast<unsigned char *>(ptr);
        ds.ready = true;
    }
    if (!(ds.tables_valid && ds.p == p && ds.f == f % p && ds.n == n)) {
        ds.tables_valid = false;
        HostPlan hp;
        FCIRC_TRY(build_host_plan(p, f, n, hp));
        FCIRC_TRY(upload_tables(ds.base, hp, ds.t, s));
        hp.U.clear(); hp.Ui.clear(); hp.sig.clear(); hp.ftw.clear(); hp.fitw.clear();
        hp.g.clear(); hp.gi.clear(); hp.gl.clear(); hp.gil.clear(); hp.rho.clear();
        ds.h = hp;
        ds.p = p;
        ds.f = f % p;
        ds.n = n;
        ds.tables_valid = true;
    }
    const HostPlan &h = ds.h;
    const DevTables &t = ds.t;

    TileJob tj;
    tj.sig = t.sig;
    tj.rho = t.rho;
    tj.U = t.U;
    tj.Ui = t.Ui;
    tj.p = p;
    tj.pinv = h.pinv;
    const Src sa{a, n, SRC_U32, 1, h.kt}, sx{x, n, SRC_U32, 0, Tw{0, 0}};
    TileParams tp;
    tp.N = n;
    tp.logT = h.logT;
    tp.D = h.D;
    if (h.k == 0) {
        tj.a = sa;
        tj.x = sx;
        tj.dst = c;
        tj.store_lazy = 0;
        tp.job[0] = tj;
        FCIRC_TRY(fast_tile_ok(h.logT) ? launch_tile_fast(tp, 1, 1, s) : launch_tile(tp, 1, 1, s));
        return FCIRC_OK;
    }
    uint32_t *xs = reinterpret_cast<uint32_t *>(ds.base);   // the vector side's intermediate
    const int lf = h.k;
    if (fast_col_ok(lf, h.m - lf)) {
        ColFwdParams fp{};
        fp.job[0] = ColFwdJob{sa, c, t.g, p, 0, 0, t.gl};
        fp.job[1] = ColFwdJob{sx, xs, t.g, p, 1, 0, t.gl};
        fp.jobs_per_cta = 1;
        fp.N = (uint32_t)n;
        fp.logn = h.m;
        fp.l0 = 0;
        fp.l1 = lf;
        for (int st = 0; st < 3; ++st) fp.stage_off[st] = h.stage_off[0][st];
        FCIRC_TRY(launch_colfwd(fp, 2, s));
    } else {
        StrFwdParams fp{};
        fp.job[0] = StrFwdJob{sa, c, t.ftw, p, 0};
        fp.job[1] = StrFwdJob{sx, xs, t.ftw, p, 1};
        fp.N = n;
        fp.logn = h.m;
        fp.l0 = 0;
        fp.l1 = lf;
        fp.logW = 2;
        FCIRC_TRY(launch_strided_fwd(fp, 2, s));
    }
    tj.a = Src{c, n, SRC_U32, 0, Tw{0, 0}};
    tj.x = Src{xs, n, SRC_U32, 0, Tw{0, 0}};
    tj.dst = c;
    tj.store_lazy = 1;
    tp.job[0] = tj;
    FCIRC_TRY(fast_tile_ok(h.logT) ? launch_tile_fast(tp, (uint64_t)1 << h.k, 1, s)
                                   : launch_tile(tp, (uint64_t)1 << h.k, 1, s));
    if (fast_col_ok(lf, h.m - lf)) {
        ColInvParams ip{};
        ip.job[0] = ColInvJob{c, c, t.gi, p, t.gil};
        ip.nprime = 1;
        ip.N = (uint32_t)n;
        ip.logn = h.m;
        ip.l0 = 0;
        ip.l1 = lf;
        for (int st = 0; st < 3; ++st) ip.stage_off[st] = h.stage_off[0][st];
        ip.epi = EPI_CANON;
        FCIRC_TRY(launch_colinv(ip, s));
    } else {
        StrInvParams ip{};
        ip.job[0] = StrInvJob{c, c, t.fitw, p};
        ip.nprime = 1;
        ip.N = n;
        ip.logn = h.m;
        ip.l0 = 0;
        ip.l1 = lf;
        ip.logW = 2;
        ip.epi = EPI_CANON;
        FCIRC_TRY(launch_strided_inv(ip, s));
    }
    return FCIRC_OK;
}
