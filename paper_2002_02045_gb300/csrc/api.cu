// C ABI entry points of libpertgb (declared in include/pertgb.h): argument
// checks, host/device staging, memory ownership and the call sequences of the
// interpolation, rates, collision and RK4 paths.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "../../include/pertgb_diag.h"

using namespace pgb;

namespace {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Input buffer that is host or device: device pointers are used in place,
// host pointers are copied to a stream-ordered temporary.
template <typename T>
struct In {
    const T *dev = nullptr;
    T *tmp = nullptr;
    pgb_ctx *c = nullptr;
    pgb_status init(pgb_ctx *ctx, const T *p, size_t n) {
        c = ctx;
        if (n == 0) return PGB_OK;
        if (!p) {
            c->err = "null input pointer";
            return PGB_EINVAL;
        }
        if (is_device_ptr(p)) {
            dev = p;
            return PGB_OK;
        }
        PGB_CUDA_TRY(c, dev_malloc_async((void **)&tmp, n * sizeof(T), c->stream));
        PGB_CUDA_TRY(c, cudaMemcpyAsync(tmp, p, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        dev = tmp;
        return PGB_OK;
    }
    ~In() {
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
};

// Output buffer that is host or device: host outputs are produced in a
// temporary and copied back by finish(), which synchronises the stream.
template <typename T>
struct Out {
    T *dev = nullptr;
    T *host = nullptr;
    T *tmp = nullptr;
    size_t n = 0;
    pgb_ctx *c = nullptr;
    pgb_status init(pgb_ctx *ctx, T *p, size_t count) {
        c = ctx;
        n = count;
        if (!p) return PGB_OK;
        if (is_device_ptr(p)) {
            dev = p;
            return PGB_OK;
        }
        host = p;
        if (n == 0) return PGB_OK;
        PGB_CUDA_TRY(c, dev_malloc_async((void **)&tmp, n * sizeof(T), c->stream));
        dev = tmp;
        return PGB_OK;
    }
    pgb_status finish() {
        if (host && n) {
            PGB_CUDA_TRY(c, cudaMemcpyAsync(host, tmp, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
            PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        }
        return PGB_OK;
    }
    ~Out() {
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
};

// Stream-ordered temporary device array.
template <typename T>
struct Tmp {
    T *p = nullptr;
    pgb_ctx *c = nullptr;
    pgb_status alloc(pgb_ctx *ctx, size_t n) {
        c = ctx;
        if (n == 0) return PGB_OK;
        PGB_CUDA_TRY(c, dev_malloc_async((void **)&p, n * sizeof(T), c->stream));
        return PGB_OK;
    }
    ~Tmp() {
        if (p) cudaFreeAsync(p, c->stream);
    }
};

#define TRY(expr)                          \
    do {                                   \
        pgb_status _s = (expr);            \
        if (_s != PGB_OK) return _s;       \
    } while (0)

pgb_status fail(pgb_ctx *c, pgb_status s, const std::string &msg) {
    c->err = msg;
    return s;
}

using RKey = std::tuple<int, int, int>;

std::map<RKey, int> r_index(const int32_t *R, int n) {
    std::map<RKey, int> m;
    for (int i = 0; i < n; ++i) m[RKey(R[3 * i], R[3 * i + 1], R[3 * i + 2])] = i;
    return m;
}

// Interpolate bands at arbitrary points: phases -> H(k) (complex GEMM) -> Jacobi.
pgb_status bands_at(pgb_ctx *c, const double *d_pts, int64_t np, double *d_eps, double2 *d_U) {
    const int nw2 = c->nw * c->nw;
    Tmp<double2> ph, hk;
    TRY(ph.alloc(c, (size_t)np * c->nRH));
    TRY(hk.alloc(c, (size_t)np * nw2));
    TRY(launch_phase_pts(c, d_pts, np, c->d_RH, c->nRH, ph.p, false));
    prof_mark(c, PGB_PROF_BANDS);
    TRY(launch_cgemm(c, false, 1, np, nw2, c->nRH, ph.p, c->nRH, 0, c->d_H, nw2, 0, hk.p, nw2, 0));
    prof_mark(c, PGB_PROF_BANDS);
    TRY(launch_heevj(c, np, c->nw, hk.p, nullptr, d_eps, d_U));
    return PGB_OK;
}

// Bands at arbitrary points for the FP32 paths: real cos/sin Fourier sum of the
// packed Hermitian H(k), FP32 Jacobi eigenvectors, FP64-refined eigenvalues.
pgb_status bands_at_mixed(pgb_ctx *c, const double *d_pts, int64_t np, double *d_eps, float2 *d_U32,
                          double2 *d_U64) {
    if (c->nw < 2) return fail(c, PGB_EINVAL, "bands_at_mixed: needs nw >= 2");
    Tmp<double> hp;
    TRY(hp.alloc(c, (size_t)np * c->nw * c->nw));
    prof_mark(c, PGB_PROF_BANDS);
    TRY(launch_herm_sum(c, c->htH, d_pts, np, hp.p));
    prof_mark(c, PGB_PROF_BANDS);
    TRY(launch_heev_mixed(c, np, c->nw, hp.p, d_eps, d_U32, d_U64, false));
    return PGB_OK;
}

// Phonons at arbitrary points for the FP32 paths: cos/sin Fourier sum of the
// mass-scaled D(q), mixed-precision Jacobi (FP64-refined omega^2, FP32 modes).
pgb_status phonons_at_mixed(pgb_ctx *c, const double *d_pts, int64_t np, double *d_hw, double2 *d_coef) {
    const int nm2 = c->nm * c->nm;
    Tmp<double> dp, lam;
    Tmp<double2> ev;
    TRY(dp.alloc(c, (size_t)np * nm2));
    TRY(lam.alloc(c, (size_t)np * c->nm));
    TRY(ev.alloc(c, (size_t)np * nm2));
    TRY(launch_herm_sum(c, c->htD, d_pts, np, dp.p));
    TRY(launch_heev_mixed(c, np, c->nm, dp.p, lam.p, nullptr, ev.p, true));
    TRY(launch_phonon_coef(c, np, c->nm, lam.p, ev.p, c->d_mode_scale, d_hw, d_coef));
    return PGB_OK;
}

// Interpolate phonons at arbitrary points: hbar*omega and mode coefficients.
pgb_status phonons_at(pgb_ctx *c, const double *d_pts, int64_t np, double *d_hw, double2 *d_coef) {
    const int nm2 = c->nm * c->nm;
    Tmp<double2> ph, dq, ev;
    Tmp<double> lam;
    TRY(ph.alloc(c, (size_t)np * c->nRD));
    TRY(dq.alloc(c, (size_t)np * nm2));
    TRY(ev.alloc(c, (size_t)np * nm2));
    TRY(lam.alloc(c, (size_t)np * c->nm));
    TRY(launch_phase_pts(c, d_pts, np, c->d_RD, c->nRD, ph.p, false));
    TRY(launch_cgemm(c, false, 1, np, nm2, c->nRD, ph.p, c->nRD, 0, c->d_D, nm2, 0, dq.p, nm2, 0));
    TRY(launch_heevj(c, np, c->nm, dq.p, c->d_mode_scale, lam.p, ev.p));
    TRY(launch_phonon_coef(c, np, c->nm, lam.p, ev.p, c->d_mode_scale, d_hw, d_coef));
    return PGB_OK;
}

void free_grids(pgb_ctx *c) {
    dfree(&c->d_eps);
    dfree(&c->d_U);
    dfree(&c->d_U32);
    dfree(&c->d_U32T);
    dfree(&c->d_hw);
    dfree(&c->d_coef);
    dfree(&c->d_coef32);
    dfree(&c->d_coefT);
    dfree(&c->d_phq64);
    dfree(&c->d_phq32);
    if (c->d_asplit) cudaFree(c->d_asplit);
    c->d_asplit = nullptr;
    c->asplit_prec = -1;
    dfree(&c->d_polarL);
    c->has_grids = false;
}

void free_coll(pgb_ctx *c) {
    dfree(&c->d_eps_state);
    dfree(&c->d_rowptr);
    dfree(&c->d_col);
    dfree(&c->d_a);
    dfree(&c->d_b);
    dfree(&c->d_rowsum_a);
    dfree(&c->d_active_rows);
    c->nrows_active = 0;
    for (int i = 0; i < 4; ++i) dfree(&c->d_f[i]);
    for (int i = 0; i < 3; ++i) dfree(&c->d_f32[i]);
    dfree(&c->d_coo_row);
    dfree(&c->d_coo_col);
    dfree(&c->d_coo_mode);
    dfree(&c->d_coo_g2);
    free_adjoint(c);
    c->has_coll = false;
    c->nstates = c->nnz = 0;
    c->coll_elo = -1e300;
    c->coll_ehi = 1e300;
}

void free_model(pgb_ctx *c) {
    dfree(&c->d_RH);
    dfree(&c->d_RD);
    dfree(&c->d_Rge);
    dfree(&c->d_Rgp);
    dfree(&c->d_H);
    free_herm_table(&c->htH);
    free_herm_table(&c->htD);
    dfree(&c->d_D);
    dfree(&c->d_mode_scale);
    dfree(&c->d_g64);
    dfree(&c->d_g32);
    if (c->d_gsplit) cudaFree(c->d_gsplit);
    c->d_gsplit = nullptr;
    c->gsplit_prec = -1;
    dfree(&c->d_Hd);
    dfree(&c->d_polar);
    dfree(&c->d_gvec);
    c->has_lattice = false;
    c->polar = false;
    c->nG = 0;
    c->has_model = false;
}

__global__ void k_f32_to_f64(const float2 *s, double2 *d, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) d[t] = make_double2(s[t].x, s[t].y);
}

}  // namespace

namespace pgb {
namespace alloc_hook {
std::atomic<int64_t> count{0};   // device allocations requested since the library was loaded
std::atomic<int64_t> fail{-1};   // index of the allocation to refuse, or -1
}  // namespace alloc_hook

cudaError_t dev_malloc_raw(void **p, size_t bytes, cudaStream_t stream, bool async) {
    const int64_t n = alloc_hook::count.fetch_add(1);
    int64_t f = n;
    if (alloc_hook::fail.load() == n && alloc_hook::fail.compare_exchange_strong(f, -1)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return async ? cudaMallocAsync(p, bytes, stream) : cudaMalloc(p, bytes);
}

void prof_mark(pgb_ctx *c, int id) {
    if (!c->prof) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e, c->stream);
    c->prof_ev[id].push_back(e);
}

pgb_status ensure_scratch(pgb_ctx *c, size_t bytes) {
    if (bytes <= c->scratch_bytes) return PGB_OK;
    if (c->scratch) {
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    PGB_CUDA_TRY(c, dev_malloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    return PGB_OK;
}
}  // namespace pgb

// ===========================================================================
// ABI
// ===========================================================================
namespace {

// True when none of the n IEEE values at p (bit patterns of width U) has an all-ones
// exponent (inf or NaN).  Branch-free blocks, split over host threads for the
// hundreds of megabytes of a g~ table.
template <typename U, U EXP>
bool finite_block(const U *p, size_t n) {
    constexpr size_t B = 4096;
    for (size_t i0 = 0; i0 < n; i0 += B) {
        const size_t e = std::min(n, i0 + B);
        U bad = 0;
        for (size_t i = i0; i < e; ++i) bad |= (U)((p[i] & EXP) == EXP);
        if (bad) return false;
    }
    return true;
}

template <typename U, U EXP>
bool all_finite(const void *x, size_t n) {
    const U *p = static_cast<const U *>(x);
    unsigned nt = std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n < ((size_t)1 << 22)) nt = 1;
    std::vector<char> ok(nt, 1);
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) {
        const size_t a = n * t / nt, b = n * (t + 1) / nt;
        th.emplace_back([&ok, p, a, b, t] { ok[t] = finite_block<U, EXP>(p + a, b - a); });
    }
    ok[0] = finite_block<U, EXP>(p, n / nt);
    for (auto &t : th) t.join();
    return std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; });
}

}  // namespace

extern "C" {

const char *pgb_status_string(int s) {
    switch (s) {
        case PGB_OK: return "ok";
        case PGB_EINVAL: return "invalid argument";
        case PGB_ESTATE: return "call order violated";
        case PGB_ENOMEM: return "device allocation failed";
        case PGB_ECUDA: return "CUDA error";
        case PGB_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

pgb_status pgb_create(pgb_ctx **out, int device, void *cuda_stream) {
    if (!out) return PGB_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return PGB_ECUDA;
    }
    if (device < 0 || device >= n) return PGB_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PGB_ECUDA;
    pgb_ctx *c = new (std::nothrow) pgb_ctx();
    if (!c) return PGB_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return PGB_OK;
}

void pgb_destroy(pgb_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_coll(c);
    free_grids(c);
    free_model(c);
    if (c->scratch) cudaFree(c->scratch);
    if (c->d_err) cudaFree(c->d_err);
    for (auto &v : c->prof_ev)
        for (auto e : v) cudaEventDestroy(e);
    delete c;
}

const char *pgb_last_error(const pgb_ctx *c) { return c ? c->err.c_str() : "null context"; }

int64_t pgb_launch_count(const pgb_ctx *c) { return c ? c->launches : 0; }

pgb_status pgb_profile(pgb_ctx *c, int enable) {
    if (!c) return PGB_EINVAL;
    c->prof = enable != 0;
    return PGB_OK;
}

pgb_status pgb_profile_read(pgb_ctx *c, int id, double *total_ms, int64_t *launches) {
    if (!c) return PGB_EINVAL;
    if (id < 0 || id >= PGB_PROF_NKERNELS) return fail(c, PGB_EINVAL, "profile_read: unknown kernel class");
    cudaSetDevice(c->device);
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    auto &ev = c->prof_ev[id];
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        float ms = 0.f;
        PGB_CUDA_TRY(c, cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        c->prof_ms[id] += ms;
        c->prof_n[id] += 1;
    }
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    if (total_ms) *total_ms = c->prof_ms[id];
    if (launches) *launches = c->prof_n[id];
    c->prof_ms[id] = 0.0;
    c->prof_n[id] = 0;
    return PGB_OK;
}

pgb_status pgb_set_model(pgb_ctx *c, const pgb_model *m) {
    if (!c) return PGB_EINVAL;
    if (!m) return fail(c, PGB_EINVAL, "set_model: null model");
    cudaSetDevice(c->device);
    if (m->nw < 1 || m->nw > kMaxNw) return fail(c, PGB_EINVAL, "set_model: nw must be 1..16");
    if (m->nat < 1 || 3 * m->nat > kMaxNmode) return fail(c, PGB_EINVAL, "set_model: nat must be 1..5");
    if (m->nR_H < 1 || m->nR_D < 1 || m->nR_ge < 1 || m->nR_gp < 1)
        return fail(c, PGB_EINVAL, "set_model: every R list needs at least one vector");
    if (!m->mass || !m->R_H || !m->H || !m->R_D || !m->D || !m->R_ge || !m->R_gp || !m->g)
        return fail(c, PGB_EINVAL, "set_model: null array");
    const int nw = m->nw, nm = 3 * m->nat, nw2 = nw * nw, nm2 = nm * nm;
    for (int i = 0; i < m->nat; ++i)
        if (!(m->mass[i] > 0.0) || !std::isfinite(m->mass[i]))
            return fail(c, PGB_EINVAL, "set_model: masses must be positive");
    // H(-R) = H(R)^dagger
    {
        auto idx = r_index(m->R_H, m->nR_H);
        for (int r = 0; r < m->nR_H; ++r) {
            auto it = idx.find(RKey(-m->R_H[3 * r], -m->R_H[3 * r + 1], -m->R_H[3 * r + 2]));
            if (it == idx.end()) return fail(c, PGB_EINVAL, "set_model: R_H is not closed under inversion");
            const double *a = m->H + 2 * (size_t)r * nw2;
            const double *b = m->H + 2 * (size_t)it->second * nw2;
            for (int i = 0; i < nw; ++i)
                for (int j = 0; j < nw; ++j) {
                    const double ar = a[2 * (i * nw + j)], ai = a[2 * (i * nw + j) + 1];
                    const double br = b[2 * (j * nw + i)], bi = b[2 * (j * nw + i) + 1];
                    if (!std::isfinite(ar) || !std::isfinite(ai))
                        return fail(c, PGB_EINVAL, "set_model: non-finite H");
                    if (std::fabs(ar - br) > 1e-10 * (1.0 + std::fabs(ar)) ||
                        std::fabs(ai + bi) > 1e-10 * (1.0 + std::fabs(ai)))
                        return fail(c, PGB_EINVAL, "set_model: H(-R) != H(R)^dagger");
                }
        }
    }
    // D(-R) = D(R)^T
    {
        auto idx = r_index(m->R_D, m->nR_D);
        for (int r = 0; r < m->nR_D; ++r) {
            auto it = idx.find(RKey(-m->R_D[3 * r], -m->R_D[3 * r + 1], -m->R_D[3 * r + 2]));
            if (it == idx.end()) return fail(c, PGB_EINVAL, "set_model: R_D is not closed under inversion");
            const double *a = m->D + (size_t)r * nm2;
            const double *b = m->D + (size_t)it->second * nm2;
            for (int i = 0; i < nm; ++i)
                for (int j = 0; j < nm; ++j) {
                    if (!std::isfinite(a[i * nm + j])) return fail(c, PGB_EINVAL, "set_model: non-finite D");
                    if (std::fabs(a[i * nm + j] - b[j * nm + i]) > 1e-10 * (1.0 + std::fabs(a[i * nm + j])))
                        return fail(c, PGB_EINVAL, "set_model: D(-R) != D(R)^T");
                }
        }
    }
    const size_t ng = (size_t)m->nR_ge * m->nR_gp * nm * nw2;
    const bool g_ok = m->g_is_double ? all_finite<uint64_t, 0x7ff0000000000000ull>(m->g, 2 * ng)
                                     : all_finite<uint32_t, 0x7f800000u>(m->g, 2 * ng);
    if (!g_ok) return fail(c, PGB_EINVAL, "set_model: non-finite g");

    free_coll(c);
    free_grids(c);
    free_model(c);
    c->nw = nw;
    c->nat = m->nat;
    c->nm = nm;
    c->nRH = m->nR_H;
    c->nRD = m->nR_D;
    c->nRge = m->nR_ge;
    c->nRgp = m->nR_gp;
    c->nKp = m->nR_gp;
    c->mass.assign(m->mass, m->mass + m->nat);
    TRY(dalloc(c, &c->d_RH, 3 * (size_t)c->nRH));
    TRY(dalloc(c, &c->d_RD, 3 * (size_t)c->nRD));
    TRY(dalloc(c, &c->d_Rge, 3 * (size_t)c->nRge));
    TRY(dalloc(c, &c->d_Rgp, 3 * (size_t)c->nRgp));
    TRY(dalloc(c, &c->d_H, (size_t)c->nRH * nw2));
    TRY(dalloc(c, &c->d_D, (size_t)c->nRD * nm2));
    TRY(dalloc(c, &c->d_mode_scale, (size_t)nm));
    TRY(dalloc(c, &c->d_g64, ng));
    TRY(dalloc(c, &c->d_g32, ng));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_RH, m->R_H, 12 * (size_t)c->nRH, cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_RD, m->R_D, 12 * (size_t)c->nRD, cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_Rge, m->R_ge, 12 * (size_t)c->nRge, cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_Rgp, m->R_gp, 12 * (size_t)c->nRgp, cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_H, m->H, 16 * (size_t)c->nRH * nw2, cudaMemcpyHostToDevice, c->stream));
    TRY(build_herm_table(c, &c->htH, m->R_H, m->H, c->nRH, nw));
    std::vector<double> D2((size_t)2 * c->nRD * nm2, 0.0);
    for (size_t i = 0; i < (size_t)c->nRD * nm2; ++i) D2[2 * i] = m->D[i];
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_D, D2.data(), 8 * D2.size(), cudaMemcpyHostToDevice, c->stream));
    std::vector<double> sc(nm);
    for (int ka = 0; ka < nm; ++ka) sc[ka] = 1.0 / std::sqrt(m->mass[ka / 3]);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_mode_scale, sc.data(), 8 * (size_t)nm, cudaMemcpyHostToDevice, c->stream));
    {   // the mass-scaled D(R) / sqrt(M M') as complex entries, for the cos/sin form of D(q)
        std::vector<double> Ds((size_t)2 * c->nRD * nm2, 0.0);
        for (size_t r = 0; r < (size_t)c->nRD; ++r)
            for (int i = 0; i < nm; ++i)
                for (int j = 0; j < nm; ++j) Ds[2 * (r * nm2 + i * nm + j)] = m->D[r * nm2 + i * nm + j] * sc[i] * sc[j];
        TRY(build_herm_table(c, &c->htD, m->R_D, Ds.data(), c->nRD, nm));
    }
    if (m->g_is_double) {
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_g64, m->g, 16 * ng, cudaMemcpyHostToDevice, c->stream));
        TRY(launch_to_f32(c, c->d_g64, c->d_g32, (int64_t)ng));
    } else {
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_g32, m->g, 8 * ng, cudaMemcpyHostToDevice, c->stream));
        k_f32_to_f64<<<(unsigned int)((ng + 255) / 256), 256, 0, c->stream>>>(c->d_g32, c->d_g64, (int64_t)ng);
        PGB_LAUNCH_CHECK(c);
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // host vectors above go out of scope
    c->has_model = true;
    return PGB_OK;
}

pgb_status pgb_set_grids(pgb_ctx *c, const int kgrid[3], const int qgrid[3]) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "set_grids: call set_model first");
    if (!kgrid || !qgrid) return fail(c, PGB_EINVAL, "set_grids: null grid");
    for (int d = 0; d < 3; ++d) {
        if (kgrid[d] < 1 || qgrid[d] < 1 || kgrid[d] > 1024 || qgrid[d] > 1024)
            return fail(c, PGB_EINVAL, "set_grids: grid sizes must be 1..1024");
        if (kgrid[d] % qgrid[d] != 0) return fail(c, PGB_EINVAL, "set_grids: q grid must divide the k grid");
    }
    free_coll(c);
    free_grids(c);
    for (int d = 0; d < 3; ++d) {
        c->kg[d] = kgrid[d];
        c->qg[d] = qgrid[d];
    }
    c->Nk = (int64_t)kgrid[0] * kgrid[1] * kgrid[2];
    c->Nq = (int64_t)qgrid[0] * qgrid[1] * qgrid[2];
    const int nw2 = c->nw * c->nw, nm2 = c->nm * c->nm;
    TRY(dalloc(c, &c->d_eps, (size_t)c->Nk * c->nw));
    TRY(dalloc(c, &c->d_U, (size_t)c->Nk * nw2));
    TRY(dalloc(c, &c->d_U32, (size_t)c->Nk * nw2));
    TRY(dalloc(c, &c->d_U32T, (size_t)c->Nk * nw2));
    TRY(dalloc(c, &c->d_hw, (size_t)c->Nq * c->nm));
    TRY(dalloc(c, &c->d_coef, (size_t)c->Nq * nm2));
    TRY(dalloc(c, &c->d_coef32, (size_t)c->Nq * nm2));
    TRY(dalloc(c, &c->d_coefT, (size_t)c->Nq * nm2));
    {   // bands on the k grid (chunks bound the phase-table size)
        const int64_t chunk = 1 << 16;
        Tmp<double2> ph, hk;
        TRY(ph.alloc(c, (size_t)std::min<int64_t>(chunk, c->Nk) * c->nRH));
        TRY(hk.alloc(c, (size_t)std::min<int64_t>(chunk, c->Nk) * nw2));
        std::vector<int32_t> idx;
        Tmp<int32_t> didx;
        TRY(didx.alloc(c, (size_t)std::min<int64_t>(chunk, c->Nk)));
        for (int64_t k0 = 0; k0 < c->Nk; k0 += chunk) {
            const int64_t nk = std::min<int64_t>(chunk, c->Nk - k0);
            idx.resize(nk);
            for (int64_t i = 0; i < nk; ++i) idx[i] = (int32_t)(k0 + i);
            PGB_CUDA_TRY(c, cudaMemcpyAsync(didx.p, idx.data(), 4 * nk, cudaMemcpyHostToDevice, c->stream));
            TRY(launch_phase_grid(c, c->kg, didx.p, nk, c->d_RH, c->nRH, ph.p, false));
            TRY(launch_cgemm(c, false, 1, nk, nw2, c->nRH, ph.p, c->nRH, 0, c->d_H, nw2, 0, hk.p, nw2, 0));
            TRY(launch_heevj(c, nk, c->nw, hk.p, nullptr, c->d_eps + k0 * c->nw, c->d_U + k0 * nw2));
            PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        }
    }
    {   // phonons on the q grid
        Tmp<double2> ph, dq, ev;
        Tmp<double> lam;
        TRY(ph.alloc(c, (size_t)c->Nq * c->nRD));
        TRY(dq.alloc(c, (size_t)c->Nq * nm2));
        TRY(ev.alloc(c, (size_t)c->Nq * nm2));
        TRY(lam.alloc(c, (size_t)c->Nq * c->nm));
        TRY(launch_phase_grid(c, c->qg, nullptr, c->Nq, c->d_RD, c->nRD, ph.p, false));
        TRY(launch_cgemm(c, false, 1, c->Nq, nm2, c->nRD, ph.p, c->nRD, 0, c->d_D, nm2, 0, dq.p, nm2, 0));
        TRY(launch_heevj(c, c->Nq, c->nm, dq.p, c->d_mode_scale, lam.p, ev.p));
        TRY(launch_phonon_coef(c, c->Nq, c->nm, lam.p, ev.p, c->d_mode_scale, c->d_hw, c->d_coef));
    }
    TRY(launch_to_f32(c, c->d_U, c->d_U32, c->Nk * nw2));
    TRY(launch_transpose_u(c));
    {   // energy shift of the FP32 tables: every shifted band energy >= 1 eV
        std::vector<double> e((size_t)c->Nk * c->nw);
        PGB_CUDA_TRY(c, cudaMemcpyAsync(e.data(), c->d_eps, 8 * e.size(), cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        double lo = e.empty() ? 0.0 : e[0];
        for (double x : e) lo = std::min(lo, x);
        c->eps_ref = std::floor(lo) - 1.0;
    }
    TRY(launch_to_f32(c, c->d_coef, c->d_coef32, c->Nq * nm2));
    TRY(launch_transpose_coef(c));
    c->has_grids = true;
    const pgb_status pst = polar_grid_table(c);
    if (pst != PGB_OK) {
        c->has_grids = false;
        return pst;
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status pgb_set_lattice(pgb_ctx *c, const double lattice[9], const double *tau) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "set_lattice: call set_model first");
    if (!lattice || !tau) return fail(c, PGB_EINVAL, "set_lattice: null pointer");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(lattice[i])) return fail(c, PGB_EINVAL, "set_lattice: non-finite lattice");
    for (int i = 0; i < 3 * c->nat; ++i)
        if (!std::isfinite(tau[i])) return fail(c, PGB_EINVAL, "set_lattice: non-finite tau");
    const double *a = lattice;
    // reciprocal rows b_i = 2 pi (a_j x a_k) / (a_1 . (a_2 x a_3))
    auto cross = [](const double *u, const double *v, double *w) {
        w[0] = u[1] * v[2] - u[2] * v[1];
        w[1] = u[2] * v[0] - u[0] * v[2];
        w[2] = u[0] * v[1] - u[1] * v[0];
    };
    double x23[3], x31[3], x12[3];
    cross(a + 3, a + 6, x23);
    cross(a + 6, a + 0, x31);
    cross(a + 0, a + 3, x12);
    const double vol = a[0] * x23[0] + a[1] * x23[1] + a[2] * x23[2];
    if (!(std::fabs(vol) > 1e-12)) return fail(c, PGB_EINVAL, "set_lattice: singular lattice");
    for (int d = 0; d < 3; ++d) {
        c->rec[d] = 2 * kPi * x23[d] / vol;
        c->rec[3 + d] = 2 * kPi * x31[d] / vol;
        c->rec[6 + d] = 2 * kPi * x12[d] / vol;
    }
    for (int i = 0; i < 9; ++i) c->lat[i] = lattice[i];
    c->omega = std::fabs(vol);
    c->tau.assign(tau, tau + 3 * c->nat);
    TRY(build_velocity_tables(c));
    c->has_lattice = true;
    if (c->polar) {   // atom positions enter the long-range term
        std::vector<double> zs(c->zstar);
        std::vector<double> e(c->eps_inf, c->eps_inf + 9);
        TRY(pgb_set_polar(c, zs.data(), e.data(), c->ewald_lambda));
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status pgb_set_polar(pgb_ctx *c, const double *zstar, const double eps_inf[9], double lambda) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_lattice) return fail(c, PGB_ESTATE, "set_polar: call set_lattice first");
    if (zstar) {   // arguments are checked before any state changes
        if (!eps_inf) return fail(c, PGB_EINVAL, "set_polar: null eps_inf");
        for (int i = 0; i < 9 * c->nat; ++i)
            if (!std::isfinite(zstar[i])) return fail(c, PGB_EINVAL, "set_polar: non-finite Z*");
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (!std::isfinite(eps_inf[3 * i + j]) ||
                    std::fabs(eps_inf[3 * i + j] - eps_inf[3 * j + i]) > 1e-12 * (1.0 + std::fabs(eps_inf[3 * i + j])))
                    return fail(c, PGB_EINVAL, "set_polar: eps_inf must be symmetric and finite");
        {   // positive definite: leading principal minors
            const double *e = eps_inf;
            const double m1 = e[0], m2 = e[0] * e[4] - e[1] * e[3];
            const double m3 = e[0] * (e[4] * e[8] - e[5] * e[7]) - e[1] * (e[3] * e[8] - e[5] * e[6]) +
                              e[2] * (e[3] * e[7] - e[4] * e[6]);
            if (!(m1 > 0 && m2 > 0 && m3 > 0))
                return fail(c, PGB_EINVAL, "set_polar: eps_inf must be positive definite");
        }
        if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(c, PGB_EINVAL, "set_polar: need Lambda > 0");
        if (c->nRgp + c->nm > 4096) return fail(c, PGB_EINVAL, "set_polar: too many R_p vectors");
    }
    // every cached q table depends on the long-range columns; until the new term
    // is complete the context is non-polar
    dfree(&c->d_phq64);
    dfree(&c->d_phq32);
    if (c->d_asplit) {
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->d_asplit);
        c->d_asplit = nullptr;
    }
    c->asplit_prec = -1;
    dfree(&c->d_polarL);
    c->polar = false;
    c->nKp = c->nRgp;
    if (!zstar) return PGB_OK;
    for (int i = 0; i < 9; ++i) c->eps_inf[i] = eps_inf[i];
    c->ewald_lambda = lambda;
    c->zstar.assign(zstar, zstar + 9 * c->nat);
    std::vector<double> pol(c->tau);
    pol.insert(pol.end(), zstar, zstar + 9 * c->nat);
    TRY(dalloc(c, &c->d_polar, pol.size()));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_polar, pol.data(), 8 * pol.size(), cudaMemcpyHostToDevice, c->stream));
    std::vector<int32_t> gv = ewald_candidates(c->lat, c->eps_inf, lambda);
    c->nG = (int)(gv.size() / 3);
    TRY(dalloc(c, &c->d_gvec, gv.size()));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_gvec, gv.data(), 4 * gv.size(), cudaMemcpyHostToDevice, c->stream));
    c->polar = true;
    c->nKp = c->nRgp + c->nm;
    const pgb_status st = polar_grid_table(c);
    if (st != PGB_OK) {
        c->polar = false;
        c->nKp = c->nRgp;
        dfree(&c->d_polarL);
        return st;
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // host vectors above go out of scope
    return PGB_OK;
}

pgb_status pgb_long_range_g(pgb_ctx *c, const double *qpts, int64_t nq, double *out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "long_range_g: call set_model first");
    if (nq < 0) return fail(c, PGB_EINVAL, "long_range_g: negative nq");
    if (nq == 0) return PGB_OK;
    if (!qpts || !out) return fail(c, PGB_EINVAL, "long_range_g: null pointer");
    In<double> Q;
    TRY(Q.init(c, qpts, 3 * (size_t)nq));
    Out<double> O;
    TRY(O.init(c, out, 2 * (size_t)nq * c->nm));
    if (!c->polar)
        PGB_CUDA_TRY(c, cudaMemsetAsync(O.dev, 0, 16 * (size_t)nq * c->nm, c->stream));
    else
        TRY(launch_ewald_pts(c, Q.dev, nq, O.dev, c->nm, 0, false));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TRY(O.finish());
    return PGB_OK;
}

pgb_status pgb_get_grid_energies(pgb_ctx *c, double *eps, double *hw) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) return fail(c, PGB_ESTATE, "get_grid_energies: call set_grids first");
    if (eps)
        PGB_CUDA_TRY(c, cudaMemcpyAsync(eps, c->d_eps, 8 * (size_t)c->Nk * c->nw, cudaMemcpyDefault, c->stream));
    if (hw)
        PGB_CUDA_TRY(c, cudaMemcpyAsync(hw, c->d_hw, 8 * (size_t)c->Nq * c->nm, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status pgb_window(pgb_ctx *c, double lo, double hi, int32_t *k_idx_out, int64_t *n_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) return fail(c, PGB_ESTATE, "window: call set_grids first");
    if (!k_idx_out || !n_out) return fail(c, PGB_EINVAL, "window: null output");
    Tmp<int32_t> flag;
    TRY(flag.alloc(c, (size_t)c->Nk));
    TRY(launch_window(c, c->d_eps, c->Nk, c->nw, lo, hi, flag.p));
    std::vector<int32_t> h(c->Nk);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(h.data(), flag.p, 4 * (size_t)c->Nk, cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> list;
    for (int64_t k = 0; k < c->Nk; ++k)
        if (h[k]) list.push_back((int32_t)k);
    *n_out = (int64_t)list.size();
    if (!list.empty()) {
        PGB_CUDA_TRY(c, cudaMemcpyAsync(k_idx_out, list.data(), 4 * list.size(), cudaMemcpyDefault, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return PGB_OK;
}

pgb_status pgb_interpolate_g(pgb_ctx *c, const double *kpts, int64_t nk, const double *qpts, int64_t nq,
                             int precision, int out_mode, double *out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "interpolate_g: call set_model first");
    if (nk < 0 || nq < 0) return fail(c, PGB_EINVAL, "interpolate_g: negative size");
    if (precision < PGB_FP64 || precision > PGB_TC_BF16X3)
        return fail(c, PGB_EINVAL, "interpolate_g: unknown precision");
    if (out_mode != PGB_G2_FULL && out_mode != PGB_G_ABS)
        return fail(c, PGB_EINVAL, "interpolate_g: unknown out_mode");
    if (!out && nk * nq > 0) return fail(c, PGB_EINVAL, "interpolate_g: null output");
    if (nk == 0 || nq == 0) return PGB_OK;
    const bool tcp = precision == PGB_TC_TF32X3 || precision == PGB_TC_BF16X3;
    const bool tf32 = precision == PGB_TC_TF32X3;
    const bool f32 = precision != PGB_FP64;
    const int nw = c->nw, nm = c->nm, nw2 = nw * nw, nm2 = nm * nm;
    const int64_t ncol = (int64_t)nm * nw2, npair = nk * nq;
    // tensor-core q-sum: columns zero-padded to whole 96-column tiles
    const int64_t ldc = tcp ? (ncol + 95) / 96 * 96 : ncol;
    if (tcp && (nk > 65535 || (nq + 127) / 128 > 65535))
        return fail(c, PGB_EINVAL, "interpolate_g: tensor-core forms take at most 65535 k and 65535*128 q per call");
    const size_t es = f32 ? sizeof(float2) : sizeof(double2);
    In<double> K, Q;
    TRY(K.init(c, kpts, 3 * (size_t)nk));
    TRY(Q.init(c, qpts, 3 * (size_t)nq));
    const size_t full = (size_t)npair * nm * nw2;
    Out<double> O;
    TRY(O.init(c, out, out_mode == PGB_G2_FULL ? full : (size_t)npair * nm));
    // bands at k and k+q, phonons at q (FP64)
    Tmp<double> eps_k, eps_kq, hw_q;
    Tmp<double2> U_k, U_kq, coef_q;
    Tmp<double> kq;
    TRY(eps_k.alloc(c, (size_t)nk * nw));
    TRY(U_k.alloc(c, (size_t)nk * nw2));
    TRY(kq.alloc(c, 3 * (size_t)npair));
    TRY(eps_kq.alloc(c, (size_t)npair * nw));
    TRY(U_kq.alloc(c, (size_t)npair * nw2));
    TRY(hw_q.alloc(c, (size_t)nq * nm));
    TRY(coef_q.alloc(c, (size_t)nq * nm2));
    TRY(bands_at(c, K.dev, nk, eps_k.p, U_k.p));
    TRY(launch_kplusq_pts(c, K.dev, nk, Q.dev, nq, kq.p));
    TRY(bands_at(c, kq.p, npair, eps_kq.p, U_kq.p));
    TRY(phonons_at(c, Q.dev, nq, hw_q.p, coef_q.p));
    Tmp<float2> U_k32, U_kq32, coef_q32;
    const void *Uk = U_k.p, *Ukq = U_kq.p, *cf = coef_q.p;
    if (f32) {
        TRY(U_k32.alloc(c, (size_t)nk * nw2));
        TRY(U_kq32.alloc(c, (size_t)npair * nw2));
        TRY(coef_q32.alloc(c, (size_t)nq * nm2));
        TRY(launch_to_f32(c, U_k.p, U_k32.p, nk * nw2));
        TRY(launch_to_f32(c, U_kq.p, U_kq32.p, npair * nw2));
        TRY(launch_to_f32(c, coef_q.p, coef_q32.p, nq * nm2));
        Uk = U_k32.p;
        Ukq = U_kq32.p;
        cf = coef_q32.p;
    }
    // g: Re-sum (GEMM), fold U(k), Rp-sum (batched GEMM), epilogue.  The split
    // precisions follow pgb_scattering_rates: BF16x3 takes the R_e sum on the
    // tensor cores (when its columns tile by 96), TF32x3 the FP32 SIMT one; both
    // take the R_p sum on the tensor cores from phases split hi/lo in FP64.
    const bool tc_rsum = tcp && !tf32 && ((int64_t)c->nRgp * ncol) % 96 == 0;
    Tmp<char> phk, S1, G, phq, C, fullbuf, Asplit, Bsplit, Ak;
    const int64_t nrow = (int64_t)c->nKp * ncol;
    const int64_t nrowS = (int64_t)c->nRgp * ncol;   // g(k, R_p) rows before the long-range rows
    TRY(phk.alloc(c, (size_t)nk * c->nRge * (tcp ? sizeof(double2) : es)));
    TRY(S1.alloc(c, (size_t)nk * nrow * es));
    TRY(G.alloc(c, (size_t)nk * nrow * es));
    TRY(phq.alloc(c, (size_t)nq * c->nKp * (tcp ? sizeof(double2) : es)));
    TRY(C.alloc(c, (size_t)npair * ldc * es));
    if (tcp) {
        if (!c->d_err) PGB_CUDA_TRY(c, dev_malloc((void **)&c->d_err, sizeof(int)));
        PGB_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    }
    const void *g = f32 ? (const void *)c->d_g32 : (const void *)c->d_g64;
    if (tc_rsum) {
        const int KpE = tc_kpad(c->nRge);
        const size_t tes = tf32 ? 4 : 2;
        if (c->gsplit_prec != precision) {
            if (c->d_gsplit) {
                PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
                cudaFree(c->d_gsplit);
                c->d_gsplit = nullptr;
            }
            c->gsplit_prec = -1;
            PGB_CUDA_TRY(c, dev_malloc(&c->d_gsplit, (size_t)4 * nrowS * KpE * tes));
            TRY(launch_split_gT(c, tf32, c->nRge, nrowS, KpE, c->d_g64, c->d_gsplit));
            c->gsplit_prec = precision;
        }
        TRY(Ak.alloc(c, (size_t)4 * nk * KpE * tes));
        TRY(launch_phase_pts(c, K.dev, nk, c->d_Rge, c->nRge, phk.p, false));
        TRY(launch_split_table(c, tf32, nk, c->nRge, c->nRge, KpE, (const double2 *)phk.p, Ak.p));
        TRY(launch_tc_qsum(c, tf32, 1, nk, (int)nrowS, KpE, Ak.p, c->d_gsplit, (float2 *)S1.p, c->d_err));
    } else {
        TRY(launch_phase_pts(c, K.dev, nk, c->d_Rge, c->nRge, phk.p, f32));
        TRY(launch_cgemm(c, f32, 1, nk, nrowS, c->nRge, phk.p, c->nRge, 0, g, nrowS, 0, S1.p, nrowS, 0));
    }
    TRY(launch_fold_u(c, f32, nk, nullptr, c->nRgp, nm, nw, S1.p, Uk, G.p));
    if (tcp) {
        const int Kp = tc_kpad(c->nKp);
        const size_t tes = tf32 ? 4 : 2;
        TRY(Asplit.alloc(c, (size_t)4 * nq * Kp * tes));
        TRY(Bsplit.alloc(c, (size_t)nk * 4 * ldc * Kp * tes));
        TRY(launch_qtable_pts(c, Q.dev, nq, phq.p, false));
        TRY(launch_split_table(c, tf32, nq, c->nKp, c->nKp, Kp, (const double2 *)phq.p, Asplit.p));
        TRY(launch_split_g(c, tf32, nk, c->nKp, (int)ncol, Kp, G.p, Bsplit.p, (int)ldc));
        TRY(launch_tc_qsum(c, tf32, nk, nq, (int)ldc, Kp, Asplit.p, Bsplit.p, (float2 *)C.p, c->d_err));
    } else {
        TRY(launch_qtable_pts(c, Q.dev, nq, phq.p, f32));
        TRY(launch_cgemm(c, f32, nk, nq, ncol, c->nKp, phq.p, c->nKp, 0, G.p, ncol, nrow, C.p, ncol, nq * ncol));
    }
    double *fullp = O.dev;
    if (out_mode == PGB_G_ABS) {
        TRY(fullbuf.alloc(c, full * sizeof(double)));
        fullp = (double *)fullbuf.p;
    }
    GArgs ga;
    ga.nk = nk;
    ga.nq = nq;
    ga.nw = nw;
    ga.nm = nm;
    ga.C = C.p;
    ga.ldc = ldc;
    ga.Ukq = Ukq;
    ga.coef = cf;
    ga.out_mode = out_mode;
    ga.out = fullp;
    TRY(launch_g_epilogue(c, f32, ga));
    if (out_mode == PGB_G_ABS) TRY(launch_g_abs(c, npair, nm, nw, fullp, O.dev));
    if (tcp) {
        int herr = 0;
        PGB_CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (herr) return fail(c, PGB_ETIMEOUT, "interpolate_g: a tensor-core pipeline wait ran out (bits " +
                                                   std::to_string(herr) + ")");
    }
    TRY(O.finish());
    return PGB_OK;
}

pgb_status pgb_scattering_rates(pgb_ctx *c, const int32_t *k_idx, int64_t nk, double T, double mu, double sigma,
                                int precision, double *gamma_out, double *gamma_mode_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) return fail(c, PGB_ESTATE, "scattering_rates: call set_grids first");
    if (nk < 0) return fail(c, PGB_EINVAL, "scattering_rates: negative nk");
    if (!(T > 0.0) || !(sigma > 0.0) || !std::isfinite(mu))
        return fail(c, PGB_EINVAL, "scattering_rates: need T > 0, sigma > 0, finite mu");
    if (precision < PGB_FP64 || precision > PGB_TC_BF16X3)
        return fail(c, PGB_EINVAL, "scattering_rates: unknown precision");
    const bool tcp = precision == PGB_TC_TF32X3 || precision == PGB_TC_BF16X3;
    const bool tf32 = precision == PGB_TC_TF32X3;
    if (nk == 0) return PGB_OK;
    if (!gamma_out) return fail(c, PGB_EINVAL, "scattering_rates: null gamma_out");
    const bool f32 = precision != PGB_FP64;
    const int nw = c->nw, nm = c->nm, nw2 = nw * nw;
    const int64_t ncol = (int64_t)nm * nw2, nrow = (int64_t)c->nKp * ncol, nrowS = (int64_t)c->nRgp * ncol;
    const size_t es = f32 ? sizeof(float2) : sizeof(double2);
    const int Kp = tc_kpad(c->nKp);
    const size_t tes = tf32 ? 4 : 2;

    // k list: validate on the host
    std::vector<int32_t> hk(nk);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(hk.data(), k_idx, 4 * (size_t)nk, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < nk; ++i)
        if (hk[i] < 0 || hk[i] >= c->Nk) return fail(c, PGB_EINVAL, "scattering_rates: k index out of range");
    Tmp<int32_t> dk;
    TRY(dk.alloc(c, (size_t)nk));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(dk.p, hk.data(), 4 * (size_t)nk, cudaMemcpyHostToDevice, c->stream));

    Out<double> Gm, Gmm;
    TRY(Gm.init(c, gamma_out, (size_t)nk * nw));
    TRY(Gmm.init(c, gamma_mode_out, (size_t)nk * nm * nw));

    // q-grid phase table exp(i q.Rp), kept for later calls
    void *phq = f32 ? (void *)c->d_phq32 : (void *)c->d_phq64;
    if (!phq) {
        if (f32) {
            TRY(dalloc(c, &c->d_phq32, (size_t)c->Nq * c->nKp));
            phq = c->d_phq32;
        } else {
            TRY(dalloc(c, &c->d_phq64, (size_t)c->Nq * c->nKp));
            phq = c->d_phq64;
        }
        TRY(launch_qtable_grid(c, nullptr, c->Nq, phq, f32));
    }

    const int per = nm * nw;
    const bool fused = tcp && tc_fused_supported(nw, nm);
    // other shapes on the tensor cores: columns padded to whole 96-column tiles, the
    // q-sum in q slabs small enough to stay in L2 (kSlabBytes) until the epilogue
    // has read them
    const int64_t ldc = (ncol + 95) / 96 * 96;
    constexpr int64_t kSlabBytes = (int64_t)64 << 20;
    // BF16x3: the R_e sum on the tensor cores too (k_tc_qsum with the batch's k phases as A
    // and the split, transposed g~ as B) whenever its column count tiles by 96.  TF32x3 keeps
    // the FP32 SIMT R_e sum: a second TF32x3 sum put Gamma 1.3e-5 from the oracle on the
    // reduced fcc case, outside that path's 1e-5 bound.
    const bool tc_rsum = tcp && !tf32 && nrowS % 96 == 0;
    const int KpE = tc_kpad(c->nRge);
    const int qpb = std::max(1, 256 / nw);
    const int qiters = 8;
    const int wqc = 8;    // q-points per task of the warp epilogue (tensor-core slabs, and the FP32 form)
    // The FP32 form takes the warp epilogue when a row holds at least 96 (nu, m) combos: 16 bands x
    // 15 modes 42.6 -> 23.9 ms; with 8 bands x 6 modes (48 combos, a quarter of the lanes idle) the
    // thread-per-(q, n) epilogue was 10 % faster over the whole pass.
    const bool f32_warp = f32 && !tcp && nm * nw >= 96;
    const int64_t nqblk = fused ? (c->Nq + 127) / 128
                          : (tcp || f32_warp) ? (c->Nq + wqc - 1) / wqc
                                              : (c->Nq + (int64_t)qpb * qiters - 1) / ((int64_t)qpb * qiters);
    // scratch carve-up, every piece 256-byte aligned (TMA and vector loads)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    int64_t nbmax = 0;
    size_t o_S1 = 0, o_G = 0, o_C = 0, o_part = 0, o_gm = 0, o_B = 0, o_Ak = 0, total = 0;
    auto layout = [&](int64_t nbm) {
        o_S1 = al((size_t)nbm * c->nRge * es);
        o_G = o_S1 + al((size_t)nbm * nrow * es);
        o_C = o_G + al((size_t)nbm * nrow * es);
        o_part = o_C + (fused ? 0 : tcp ? al((size_t)kSlabBytes) : al((size_t)nbm * c->Nq * ncol * es));
        o_gm = o_part + al((size_t)nbm * nqblk * per * sizeof(double));
        o_B = o_gm + al((size_t)nbm * per * sizeof(double));
        o_Ak = o_B + (tcp ? al((size_t)nbm * (fused ? 6 * ncol : 4 * ldc) * Kp * tes) : 0);
        total = o_Ak + (tc_rsum ? al((size_t)nbm * 4 * KpE * tes) : 0);
    };
    layout(1);
    const size_t budget = (size_t)4 << 30;
    nbmax = std::max<int64_t>(1, (int64_t)(budget / total));
    nbmax = std::min<int64_t>(nbmax, std::min<int64_t>(nk, 65535));
    if (tcp && !fused)   // a slab holds at least 128 q-points of every k of the batch
        nbmax = std::max<int64_t>(1, std::min<int64_t>(nbmax, kSlabBytes / (128 * ldc * (int64_t)sizeof(float2))));
    layout(nbmax);
    TRY(ensure_scratch(c, total));
    char *base = (char *)c->scratch;
    char *phk = base;
    char *S1 = base + o_S1;
    char *G = base + o_G;
    char *Cb = base + o_C;
    double *partial = (double *)(base + o_part);
    double *gmode_tmp = (double *)(base + o_gm);
    void *Bsplit = base + o_B;
    void *Ak = base + o_Ak;
    Tmp<double> focc, nbe;
    Tmp<float> eps32, hw32;
    TRY(focc.alloc(c, (size_t)c->Nk * nw));
    TRY(eps32.alloc(c, (size_t)c->Nk * nw));
    TRY(nbe.alloc(c, (size_t)c->Nq * nm));
    TRY(hw32.alloc(c, (size_t)c->Nq * nm));
    TRY(launch_occ_tables(c, T, mu, focc.p, eps32.p, nbe.p, hw32.p));
    Tmp<float2> ehl, whl;
    Tmp<float> focc32, nbe32;
    if (fused) {
        TRY(ehl.alloc(c, (size_t)c->Nk * nw));
        TRY(focc32.alloc(c, (size_t)c->Nk * nw));
        TRY(whl.alloc(c, (size_t)c->Nq * nm));
        TRY(nbe32.alloc(c, (size_t)c->Nq * nm));
        TRY(launch_fp32_tables(c, focc.p, nbe.p, ehl.p, focc32.p, whl.p, nbe32.p));
    }
    if (tcp) {
        if (!c->d_err) {
            PGB_CUDA_TRY(c, dev_malloc((void **)&c->d_err, sizeof(int)));
        }
        PGB_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        if (c->asplit_prec != precision) {
            if (c->d_asplit) {
                PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
                cudaFree(c->d_asplit);
                c->d_asplit = nullptr;
            }
            PGB_CUDA_TRY(c, dev_malloc(&c->d_asplit, (size_t)4 * c->Nq * Kp * tes));
            TRY(launch_split_phases(c, tf32, c->qg, c->Nq, c->d_Rgp, c->nRgp, Kp, c->d_asplit, c->d_polarL,
                                    c->polar ? nm : 0));
            c->asplit_prec = precision;
        }
    }
    if (tc_rsum && c->gsplit_prec != precision) {
        if (c->d_gsplit) {
            PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            cudaFree(c->d_gsplit);
            c->d_gsplit = nullptr;
        }
        c->gsplit_prec = -1;
        PGB_CUDA_TRY(c, dev_malloc(&c->d_gsplit, (size_t)4 * nrowS * KpE * tes));
        TRY(launch_split_gT(c, tf32, c->nRge, nrowS, KpE, c->d_g64, c->d_gsplit));
        c->gsplit_prec = precision;
    }
    const void *g = f32 ? (const void *)c->d_g32 : (const void *)c->d_g64;
    const void *U = f32 ? (const void *)c->d_U32 : (const void *)c->d_U;
    const void *cf = f32 ? (const void *)c->d_coef32 : (const void *)c->d_coef;
    const double scale = kTwoPiOverHbar / ((double)c->Nq * sigma * kSqrtPi);
    for (int64_t b0 = 0; b0 < nk; b0 += nbmax) {
        const int64_t nb = std::min<int64_t>(nbmax, nk - b0);
        const int32_t *kb = dk.p + b0;
        prof_mark(c, PGB_PROF_RSUM);
        if (tc_rsum) {
            TRY(launch_split_phases_pts(c, tf32, c->kg, kb, nb, c->d_Rge, c->nRge, KpE, Ak));
            TRY(launch_tc_qsum(c, tf32, 1, nb, (int)nrowS, KpE, Ak, c->d_gsplit, (float2 *)S1, c->d_err));
        } else {
            TRY(launch_phase_grid(c, c->kg, kb, nb, c->d_Rge, c->nRge, phk, f32));
            TRY(launch_cgemm(c, f32, 1, nb, nrowS, c->nRge, phk, c->nRge, 0, g, nrowS, 0, S1, nrowS, 0));
        }
        TRY(launch_fold_u(c, f32, nb, kb, c->nRgp, nm, nw, S1, U, G));
        prof_mark(c, PGB_PROF_RSUM);
        if (fused) {
            TRY(launch_split_g6(c, tf32, nb, c->nKp, (int)ncol, Kp, G, Bsplit));
            FusedLaunch L;
            L.nb = nb;
            L.kidx = kb;
            L.Kp = Kp;
            L.Bsplit = Bsplit;
            L.ehl = ehl.p;
            L.focc32 = focc32.p;
            L.whl = whl.p;
            L.nbe32 = nbe32.p;
            L.sigma = sigma;
            L.partial = partial;
            prof_mark(c, PGB_PROF_QSUM);
            TRY(launch_tc_rates(c, tf32, L));
            prof_mark(c, PGB_PROF_QSUM);
            TRY(launch_rates_reduce(c, nb, nqblk, nm, nw, scale, partial, Gm.dev + b0 * nw,
                                    Gmm.dev ? Gmm.dev + b0 * nm * nw : gmode_tmp));
            continue;
        }
        RatesArgs ra;
        ra.nb = nb;
        ra.kidx = kb;
        ra.Nq = c->Nq;
        for (int d = 0; d < 3; ++d) {
            ra.kg[d] = c->kg[d];
            ra.qg[d] = c->qg[d];
        }
        ra.nw = nw;
        ra.nm = nm;
        ra.C = Cb;
        ra.U = U;
        ra.coef = cf;
        ra.eps = c->d_eps;
        ra.hw = c->d_hw;
        ra.T = T;
        ra.mu = mu;
        ra.sigma = sigma;
        ra.eps32 = eps32.p;
        ra.focc = focc.p;
        ra.nbe = nbe.p;
        ra.hw32 = hw32.p;
        ra.partial = partial;
        ra.nqblk = nqblk;
        ra.qpb = qpb;
        ra.qiters = qiters;
        auto warp_args = [&](int64_t ld) {
            WarpRatesArgs wa;
            wa.nw = nw;
            wa.nm = nm;
            wa.ib = warp_rates_ib(nw, nm);
            for (int d = 0; d < 3; ++d) {
                wa.kg[d] = c->kg[d];
                wa.qg[d] = c->qg[d];
            }
            wa.qc = wqc;
            wa.nb = nb;
            wa.C = (const float2 *)Cb;
            wa.ldc = ld;
            wa.kidx = kb;
            wa.eps = c->d_eps;
            wa.eps32 = eps32.p;
            wa.U = c->d_U32;
            wa.coef = c->d_coef32;
            wa.hw = c->d_hw;
            wa.hw32 = hw32.p;
            wa.focc = focc.p;
            wa.nbe = nbe.p;
            wa.sigma = sigma;
            wa.partial = partial;
            wa.nqblk = nqblk;
            return wa;
        };
        if (tcp) {
            // q slabs: tensor-core q-sum into the L2-sized buffer, then the warp epilogue on that slab
            TRY(launch_split_g(c, tf32, nb, c->nKp, (int)ncol, Kp, G, Bsplit, (int)ldc));
            const int64_t sq = std::max<int64_t>(128, kSlabBytes / (nb * ldc * (int64_t)sizeof(float2)) / 128 * 128);
            WarpRatesArgs wa = warp_args(ldc);
            for (int64_t qs = 0; qs < c->Nq; qs += sq) {
                const int64_t nqs = std::min(sq, c->Nq - qs);
                prof_mark(c, PGB_PROF_QSUM);
                TRY(launch_tc_qsum(c, tf32, nb, nqs, (int)ldc, Kp, c->d_asplit, Bsplit, (float2 *)Cb, c->d_err, c->Nq,
                                   qs));
                prof_mark(c, PGB_PROF_QSUM);
                wa.q_off = qs;
                wa.nqs = nqs;
                wa.nch = (int)((nqs + wqc - 1) / wqc);
                wa.blk0 = qs / wqc;
                prof_mark(c, PGB_PROF_EPILOGUE);
                TRY(launch_rates_warp(c, wa));
                prof_mark(c, PGB_PROF_EPILOGUE);
            }
        } else {
            prof_mark(c, PGB_PROF_QSUM);
            TRY(launch_cgemm(c, f32, nb, c->Nq, ncol, c->nKp, phq, c->nKp, 0, G, ncol, nrow, Cb, ncol,
                             c->Nq * ncol));
            prof_mark(c, PGB_PROF_QSUM);
            prof_mark(c, PGB_PROF_EPILOGUE);
            if (f32_warp) {   // the warp epilogue over the whole q range (rows read from HBM)
                WarpRatesArgs wa = warp_args(ncol);
                wa.q_off = 0;
                wa.nqs = c->Nq;
                wa.nch = (int)((c->Nq + wqc - 1) / wqc);
                wa.blk0 = 0;
                TRY(launch_rates_warp(c, wa));
            } else {
                TRY(launch_rates_epilogue(c, f32, ra));
            }
            prof_mark(c, PGB_PROF_EPILOGUE);
        }
        TRY(launch_rates_reduce(c, nb, nqblk, nm, nw, scale, partial, Gm.dev + b0 * nw,
                                Gmm.dev ? Gmm.dev + b0 * nm * nw : gmode_tmp));
    }
    if (tcp) {
        int herr = 0;
        PGB_CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (herr) return fail(c, PGB_ETIMEOUT, "scattering_rates: a tensor-core pipeline wait ran out (bits " +
                                                   std::to_string(herr) + ")");
    }
    TRY(Gm.finish());
    TRY(Gmm.finish());
    return PGB_OK;
}

pgb_status pgb_build_collision(pgb_ctx *c, int band_lo, int band_hi, double T, double sigma, int64_t nnz,
                               const int32_t *row, const int32_t *col, const int32_t *mode, const float *g2) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) return fail(c, PGB_ESTATE, "build_collision: call set_grids first");
    for (int d = 0; d < 3; ++d)
        if (c->kg[d] != c->qg[d]) return fail(c, PGB_EINVAL, "build_collision: the q grid must equal the k grid");
    if (band_lo < 0 || band_hi > c->nw || band_lo >= band_hi)
        return fail(c, PGB_EINVAL, "build_collision: need 0 <= band_lo < band_hi <= nw");
    if (!(T > 0.0) || !(sigma > 0.0)) return fail(c, PGB_EINVAL, "build_collision: need T > 0, sigma > 0");
    if (nnz < 0 || nnz > ((int64_t)1 << 40)) return fail(c, PGB_EINVAL, "build_collision: bad nnz");
    const int nb = band_hi - band_lo;
    const int64_t ns = c->Nk * nb;
    if (ns > INT32_MAX) return fail(c, PGB_EINVAL, "build_collision: too many states");
    free_coll(c);
    In<int32_t> R, Cc, M;
    In<float> G;
    TRY(R.init(c, row, (size_t)nnz));
    TRY(Cc.init(c, col, (size_t)nnz));
    TRY(M.init(c, mode, (size_t)nnz));
    TRY(G.init(c, g2, (size_t)nnz));
    c->band_lo = band_lo;
    c->band_hi = band_hi;
    c->nstates = ns;
    c->nnz = nnz;
    // the list is kept on the device (pgb_collision_list, pgb_collision_set_g2, derivatives)
    TRY(dalloc(c, &c->d_coo_row, (size_t)nnz));
    TRY(dalloc(c, &c->d_coo_col, (size_t)nnz));
    TRY(dalloc(c, &c->d_coo_mode, (size_t)nnz));
    TRY(dalloc(c, &c->d_coo_g2, (size_t)nnz));
    if (nnz > 0) {
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_coo_row, R.dev, 4 * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_coo_col, Cc.dev, 4 * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_coo_mode, M.dev, 4 * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_coo_g2, G.dev, 4 * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
    }
    pgb_status st = launch_coll_coeffs(c, T, sigma, c->d_coo_row, c->d_coo_col, c->d_coo_mode, c->d_coo_g2, nnz, nb);
    if (st != PGB_OK) {
        std::string e = c->err;
        free_coll(c);
        c->err = e;
        return st;
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->has_coll = true;
    return PGB_OK;
}

pgb_status pgb_collision_energies(pgb_ctx *c, double *eps_state, int64_t *nstates_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "collision_energies: call build_collision first");
    if (nstates_out) *nstates_out = c->nstates;
    if (eps_state) {
        PGB_CUDA_TRY(c, cudaMemcpyAsync(eps_state, c->d_eps_state, 8 * (size_t)c->nstates, cudaMemcpyDefault,
                                        c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return PGB_OK;
}

pgb_status pgb_collision(pgb_ctx *c, const double *f, double *I_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "collision: call build_collision first");
    if (!f || !I_out) return fail(c, PGB_EINVAL, "collision: null pointer");
    In<double> F;
    TRY(F.init(c, f, (size_t)c->nstates));
    Out<double> I;
    TRY(I.init(c, I_out, (size_t)c->nstates));
    TRY(launch_f64_to_f32(c, F.dev, c->d_f32[0], c->nstates));
    TRY(launch_collision(c, F.dev, c->d_f32[0], I.dev, -1, 0.0, nullptr, nullptr, nullptr, nullptr));
    TRY(I.finish());
    return PGB_OK;
}

pgb_status pgb_step_rk4(pgb_ctx *c, double *f, double dt_fs, int64_t nsteps) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "step_rk4: call build_collision first");
    if (!f) return fail(c, PGB_EINVAL, "step_rk4: null f");
    if (nsteps < 0 || !std::isfinite(dt_fs)) return fail(c, PGB_EINVAL, "step_rk4: bad step");
    const size_t ns = (size_t)c->nstates;
    double *fd = f;
    double *tmp = nullptr;
    const bool host = !is_device_ptr(f);
    if (host) {
        PGB_CUDA_TRY(c, dev_malloc_async((void **)&tmp, 8 * ns, c->stream));
        PGB_CUDA_TRY(c, cudaMemcpyAsync(tmp, f, 8 * ns, cudaMemcpyHostToDevice, c->stream));
        fd = tmp;
    }
    const double dt = dt_fs * kFemto;
    double *acc = c->d_f[0], *f1 = c->d_f[1], *f2 = c->d_f[2];
    pgb_status st = PGB_OK;
    // states without entries are not visited by the kernel: their stage values are f
    float *g0 = c->d_f32[0], *g1 = c->d_f32[1], *g2 = c->d_f32[2];
    if (launch_f64_to_f32(c, fd, g0, (int64_t)ns) != PGB_OK ||
        cudaMemcpyAsync(f1, fd, 8 * ns, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(f2, fd, 8 * ns, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(g1, g0, 4 * ns, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(g2, g0, 4 * ns, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        st = fail(c, PGB_ECUDA, "step_rk4: stage buffer set-up");
    for (int64_t s = 0; s < nsteps && st == PGB_OK; ++s) {
        st = launch_collision(c, fd, g0, nullptr, 0, dt, acc, f1, g1, fd);
        if (st == PGB_OK) st = launch_collision(c, f1, g1, nullptr, 1, dt, acc, f2, g2, fd);
        if (st == PGB_OK) st = launch_collision(c, f2, g2, nullptr, 2, dt, acc, f1, g1, fd);
        if (st == PGB_OK) st = launch_collision(c, f1, g1, nullptr, 3, dt, acc, fd, g0, fd);
    }
    if (host) {
        if (st == PGB_OK) {
            cudaMemcpyAsync(f, tmp, 8 * ns, cudaMemcpyDeviceToHost, c->stream);
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = fail(c, PGB_ECUDA, "step_rk4: copy back");
        }
        cudaFreeAsync(tmp, c->stream);
    }
    return st;
}

pgb_status pgb_collision_set_g2(pgb_ctx *c, const float *g2) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "collision_set_g2: call build_collision first");
    const size_t n = (size_t)c->nnz;
    if (n == 0) return PGB_OK;
    In<float> G;
    TRY(G.init(c, g2, n));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_coo_g2, G.dev, 4 * n, cudaMemcpyDeviceToDevice, c->stream));
    TRY(launch_coll_values(c, c->d_coo_row, c->d_coo_col, c->d_coo_mode, c->d_coo_g2, c->nnz));
    TRY(launch_coll_rowsum(c));
    TRY(adjoint_values_changed(c));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status pgb_collision_vjp(pgb_ctx *c, const double *f, const double *lam, double *vjp_f, double *vjp_g2) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "collision_vjp: call build_collision first");
    if (!f || !lam || !vjp_f) return fail(c, PGB_EINVAL, "collision_vjp: null pointer");
    const size_t ns = (size_t)c->nstates;
    In<double> F, L;
    TRY(F.init(c, f, ns));
    TRY(L.init(c, lam, ns));
    Out<double> V, G;
    TRY(V.init(c, vjp_f, ns));
    TRY(G.init(c, vjp_g2, (size_t)c->nnz));
    TRY(collision_vjp(c, F.dev, L.dev, V.dev, G.dev));
    TRY(V.finish());
    TRY(G.finish());
    return PGB_OK;
}

pgb_status pgb_rk4_adjoint(pgb_ctx *c, const double *f0, double dt_fs, int64_t nsteps, int64_t checkpoint,
                           const double *lam_end, double *lam_0, double *dL_dg2, double *f_end) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "rk4_adjoint: call build_collision first");
    if (!f0 || !lam_end || !lam_0) return fail(c, PGB_EINVAL, "rk4_adjoint: null pointer");
    if (nsteps < 0 || !std::isfinite(dt_fs)) return fail(c, PGB_EINVAL, "rk4_adjoint: bad step");
    const size_t ns = (size_t)c->nstates;
    In<double> F, L;
    TRY(F.init(c, f0, ns));
    TRY(L.init(c, lam_end, ns));
    Out<double> L0, G, FE;
    TRY(L0.init(c, lam_0, ns));
    TRY(G.init(c, dL_dg2, (size_t)c->nnz));
    TRY(FE.init(c, f_end, ns));
    TRY(rk4_adjoint(c, F.dev, dt_fs, nsteps, checkpoint, L.dev, L0.dev, G.dev, FE.dev));
    TRY(L0.finish());
    TRY(G.finish());
    TRY(FE.finish());
    return PGB_OK;
}

pgb_status pgb_band_velocities(pgb_ctx *c, const int32_t *k_idx, int64_t nk, double *v_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids || !c->has_lattice) return fail(c, PGB_ESTATE, "band_velocities: call set_lattice and set_grids first");
    if (nk < 0) return fail(c, PGB_EINVAL, "band_velocities: negative nk");
    if (nk == 0) return PGB_OK;
    if (!k_idx || !v_out) return fail(c, PGB_EINVAL, "band_velocities: null pointer");
    std::vector<int32_t> hk(nk);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(hk.data(), k_idx, 4 * (size_t)nk, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < nk; ++i)
        if (hk[i] < 0 || hk[i] >= c->Nk) return fail(c, PGB_EINVAL, "band_velocities: k index out of range");
    Tmp<int32_t> dk;
    TRY(dk.alloc(c, (size_t)nk));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(dk.p, hk.data(), 4 * (size_t)nk, cudaMemcpyHostToDevice, c->stream));
    Out<double> V;
    TRY(V.init(c, v_out, (size_t)nk * c->nw * 3));
    TRY(band_velocities(c, dk.p, nk, V.dev));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TRY(V.finish());
    return PGB_OK;
}

pgb_status pgb_transport(pgb_ctx *c, double mu_eV, int precision, int max_iter, double tol, double *mobility_rta,
                         double *mobility, int64_t *iterations_out, double *F_out, double *tau_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "transport: build a collision list first");
    if (!c->has_lattice) return fail(c, PGB_ESTATE, "transport: call set_lattice first");
    if (!std::isfinite(mu_eV) || max_iter < 0 || !(tol >= 0.0))
        return fail(c, PGB_EINVAL, "transport: need finite mu, max_iter >= 0, tol >= 0");
    if (!mobility_rta || !mobility) return fail(c, PGB_EINVAL, "transport: null mobility output");
    const size_t ns = (size_t)c->nstates;
    Out<double> F, Tau;
    TRY(F.init(c, F_out, 3 * ns));
    TRY(Tau.init(c, tau_out, ns));
    double mr[9], mi[9];
    TRY(transport(c, mu_eV, precision, max_iter, tol, mr, mi, iterations_out, F.dev, Tau.dev));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(mobility_rta, mr, sizeof(mr), cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(mobility, mi, sizeof(mi), cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TRY(F.finish());
    TRY(Tau.finish());
    return PGB_OK;
}

pgb_status pgb_scattering_rates_mc(pgb_ctx *c, const double *kpts, int64_t nk, const double *u, int64_t nq,
                                   int sampling, double width, double T, double mu, double sigma, int precision,
                                   double *gamma_out, double *stderr_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "scattering_rates_mc: call set_model first");
    if (nk < 0 || nq < 0) return fail(c, PGB_EINVAL, "scattering_rates_mc: negative size");
    if (!(T > 0.0) || !(sigma > 0.0) || !std::isfinite(mu))
        return fail(c, PGB_EINVAL, "scattering_rates_mc: need T > 0, sigma > 0, finite mu");
    if (sampling != PGB_Q_UNIFORM && sampling != PGB_Q_CAUCHY)
        return fail(c, PGB_EINVAL, "scattering_rates_mc: unknown sampling");
    if (sampling == PGB_Q_CAUCHY && !(width > 0.0 && width <= 1.0))
        return fail(c, PGB_EINVAL, "scattering_rates_mc: the Cauchy width must lie in (0, 1]");
    if (precision != PGB_FP64 && precision != PGB_FP32 && precision != PGB_TC_TF32X3 && precision != PGB_TC_BF16X3)
        return fail(c, PGB_EINVAL, "scattering_rates_mc: unknown precision");
    if (nk == 0) return PGB_OK;
    if (nq == 0) return fail(c, PGB_EINVAL, "scattering_rates_mc: need at least one q sample");
    if (!kpts || !u || !gamma_out) return fail(c, PGB_EINVAL, "scattering_rates_mc: null pointer");
    const bool tcp = precision == PGB_TC_TF32X3 || precision == PGB_TC_BF16X3;
    const bool tf32 = precision == PGB_TC_TF32X3;
    const bool f32 = precision != PGB_FP64;   // FP32 epilogue for the FP32 and split forms
    const int nw = c->nw, nm = c->nm, nw2 = nw * nw, nm2 = nm * nm;
    const int64_t ncol = (int64_t)nm * nw2, nrow = (int64_t)c->nKp * ncol, nrowS = (int64_t)c->nRgp * ncol;
    const int64_t ldc = tcp ? (ncol + 95) / 96 * 96 : ncol;   // row stride of the q-sum result
    const int Kp = tcp ? tc_kpad(c->nKp) : 0;
    const size_t tes = tf32 ? 4 : 2;
    const size_t es = f32 ? sizeof(float2) : sizeof(double2);
    {   // uniforms must lie in [0, 1)
        std::vector<double> hu(3 * (size_t)nq);
        PGB_CUDA_TRY(c, cudaMemcpyAsync(hu.data(), u, 8 * hu.size(), cudaMemcpyDefault, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (double x : hu)
            if (!(x >= 0.0 && x < 1.0)) return fail(c, PGB_EINVAL, "scattering_rates_mc: u must lie in [0, 1)");
    }
    In<double> K, Uin;
    TRY(K.init(c, kpts, 3 * (size_t)nk));
    TRY(Uin.init(c, u, 3 * (size_t)nq));
    Out<double> Gm, Er;
    TRY(Gm.init(c, gamma_out, (size_t)nk * nw));
    TRY(Er.init(c, stderr_out, (size_t)nk * nw));
    Tmp<double> q, pinv, eps_k, acc;
    Tmp<double2> U_k;
    TRY(q.alloc(c, 3 * (size_t)nq));
    TRY(pinv.alloc(c, (size_t)nq));
    TRY(eps_k.alloc(c, (size_t)nk * nw));
    TRY(U_k.alloc(c, (size_t)nk * nw2));
    TRY(acc.alloc(c, (size_t)nk * 2 * nw));
    PGB_CUDA_TRY(c, cudaMemsetAsync(acc.p, 0, 16 * (size_t)nk * nw, c->stream));
    TRY(launch_mc_qpoints(c, nq, Uin.dev, sampling, width, q.p, pinv.p));
    Tmp<float2> U_k32;
    const void *Uk = U_k.p;
    if (f32) {
        TRY(U_k32.alloc(c, (size_t)nk * nw2));
        if (nw >= 2) {
            TRY(bands_at_mixed(c, K.dev, nk, eps_k.p, U_k32.p, nullptr));
        } else {
            TRY(bands_at(c, K.dev, nk, eps_k.p, U_k.p));
            TRY(launch_to_f32(c, U_k.p, U_k32.p, nk * nw2));
        }
        Uk = U_k32.p;
    } else {
        TRY(bands_at(c, K.dev, nk, eps_k.p, U_k.p));
    }
    // R_e sums with U(k) folded, for every k: G [nk][nKp][ncol]
    const int64_t kb = std::max<int64_t>(1, std::min<int64_t>(nk, 8));
    Tmp<char> phk, S1, G;
    TRY(phk.alloc(c, (size_t)kb * c->nRge * es));
    TRY(S1.alloc(c, (size_t)kb * nrowS * es));
    TRY(G.alloc(c, (size_t)nk * nrow * es));
    const void *g = f32 ? (const void *)c->d_g32 : (const void *)c->d_g64;
    for (int64_t k0 = 0; k0 < nk; k0 += kb) {
        const int64_t nb = std::min(kb, nk - k0);
        TRY(launch_phase_pts(c, K.dev + 3 * k0, nb, c->d_Rge, c->nRge, phk.p, f32));
        TRY(launch_cgemm(c, f32, 1, nb, nrowS, c->nRge, phk.p, c->nRge, 0, g, nrowS, 0, S1.p, nrowS, 0));
        TRY(launch_fold_u(c, f32, nb, nullptr, c->nRgp, nm, nw, S1.p,
                          (const char *)Uk + (size_t)k0 * nw2 * es, G.p + (size_t)k0 * nrow * es));
    }
    // q chunks x k batches
    const int64_t qc = std::min<int64_t>(nq, 8192);
    Tmp<double> hw_q, kq, eps_kq, partial;
    Tmp<double2> coef_q, U_kq;
    Tmp<char> phq, C, coef32, Ukq32;
    TRY(hw_q.alloc(c, (size_t)qc * nm));
    TRY(coef_q.alloc(c, (size_t)qc * nm2));
    Tmp<char> Asplit, Bsplit;
    TRY(phq.alloc(c, (size_t)qc * c->nKp * (tcp ? sizeof(double2) : es)));
    TRY(kq.alloc(c, 3 * (size_t)kb * qc));
    TRY(eps_kq.alloc(c, (size_t)kb * qc * nw));
    if (!f32 || nw < 2) TRY(U_kq.alloc(c, (size_t)kb * qc * nw2));
    TRY(C.alloc(c, (size_t)kb * qc * ldc * es));
    if (tcp) {
        TRY(Asplit.alloc(c, (size_t)4 * qc * Kp * tes));
        TRY(Bsplit.alloc(c, (size_t)kb * 4 * ldc * Kp * tes));
        if (!c->d_err) PGB_CUDA_TRY(c, dev_malloc((void **)&c->d_err, sizeof(int)));
        PGB_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    }
    TRY(partial.alloc(c, (size_t)mc_partial_count(c, kb, qc)));
    if (f32) {
        TRY(coef32.alloc(c, (size_t)qc * nm2 * sizeof(float2)));
        TRY(Ukq32.alloc(c, (size_t)kb * qc * nw2 * sizeof(float2)));
    }
    for (int64_t q0 = 0; q0 < nq; q0 += qc) {
        const int64_t nqc = std::min(qc, nq - q0);
        const double *qp = q.p + 3 * q0;
        if (f32)
            TRY(phonons_at_mixed(c, qp, nqc, hw_q.p, coef_q.p));
        else
            TRY(phonons_at(c, qp, nqc, hw_q.p, coef_q.p));
        TRY(launch_qtable_pts(c, qp, nqc, phq.p, f32 && !tcp));
        if (tcp) TRY(launch_split_table(c, tf32, nqc, c->nKp, c->nKp, Kp, (const double2 *)phq.p, Asplit.p));
        const void *cf = coef_q.p;
        if (f32) {
            TRY(launch_to_f32(c, coef_q.p, (float2 *)coef32.p, nqc * nm2));
            cf = coef32.p;
        }
        for (int64_t k0 = 0; k0 < nk; k0 += kb) {
            const int64_t nb = std::min(kb, nk - k0);
            TRY(launch_kplusq_pts(c, K.dev + 3 * k0, nb, qp, nqc, kq.p));
            const void *Ukq = U_kq.p;
            if (f32 && nw >= 2) {
                TRY(bands_at_mixed(c, kq.p, nb * nqc, eps_kq.p, (float2 *)Ukq32.p, nullptr));
                Ukq = Ukq32.p;
            } else {
                TRY(bands_at(c, kq.p, nb * nqc, eps_kq.p, U_kq.p));
                if (f32) {
                    TRY(launch_to_f32(c, U_kq.p, (float2 *)Ukq32.p, nb * nqc * nw2));
                    Ukq = Ukq32.p;
                }
            }
            if (tcp) {
                TRY(launch_split_g(c, tf32, nb, c->nKp, (int)ncol, Kp, (const float2 *)(G.p + (size_t)k0 * nrow * es),
                                   Bsplit.p, (int)ldc));
                TRY(launch_tc_qsum(c, tf32, nb, nqc, (int)ldc, Kp, Asplit.p, Bsplit.p, (float2 *)C.p, c->d_err));
            } else {
                TRY(launch_cgemm(c, f32, nb, nqc, ncol, c->nKp, phq.p, c->nKp, 0, G.p + (size_t)k0 * nrow * es,
                                 ncol, nrow, C.p, ncol, nqc * ncol));
            }
            TRY(launch_mc_epilogue(c, f32, nb, nqc, C.p, ldc, Ukq, eps_k.p + k0 * nw, eps_kq.p, hw_q.p, cf,
                                   pinv.p + q0, T, mu, sigma, partial.p, acc.p + k0 * 2 * nw));
        }
    }
    TRY(launch_mc_finish(c, nk, nq, sigma, acc.p, Gm.dev, Er.dev));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (tcp) {
        int herr = 0;
        PGB_CUDA_TRY(c, cudaMemcpy(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) return fail(c, PGB_ETIMEOUT, "scattering_rates_mc: a tensor-core pipeline wait ran out (bits " +
                                                   std::to_string(herr) + ")");
    }
    TRY(Gm.finish());
    TRY(Er.finish());
    return PGB_OK;
}

pgb_status pgb_population(pgb_ctx *c, const double *f, const double *E, int64_t nE, double *N_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "population: build a collision list first");
    if (nE < 0) return fail(c, PGB_EINVAL, "population: negative nE");
    if (nE == 0) return PGB_OK;
    if (!f || !E || !N_out) return fail(c, PGB_EINVAL, "population: null pointer");
    In<double> F, Ein;
    TRY(F.init(c, f, (size_t)c->nstates));
    TRY(Ein.init(c, E, (size_t)nE));
    Out<double> Nn;
    TRY(Nn.init(c, N_out, (size_t)nE));
    TRY(launch_population(c, F.dev, Ein.dev, nE, Nn.dev));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TRY(Nn.finish());
    return PGB_OK;
}

pgb_status pgb_diag_bands(pgb_ctx *c, const double *pts, int64_t n, double *Hk, double *eps, double *U) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, "diag_bands: call set_model first");
    if (n <= 0) return PGB_OK;
    const int nw2 = c->nw * c->nw;
    In<double> P;
    TRY(P.init(c, pts, 3 * (size_t)n));
    Tmp<double2> ph, hk, u;
    Tmp<double> e;
    TRY(ph.alloc(c, (size_t)n * c->nRH));
    TRY(hk.alloc(c, (size_t)n * nw2));
    TRY(u.alloc(c, (size_t)n * nw2));
    TRY(e.alloc(c, (size_t)n * c->nw));
    TRY(launch_phase_pts(c, P.dev, n, c->d_RH, c->nRH, ph.p, false));
    TRY(launch_cgemm(c, false, 1, n, nw2, c->nRH, ph.p, c->nRH, 0, c->d_H, nw2, 0, hk.p, nw2, 0));
    if (Hk) PGB_CUDA_TRY(c, cudaMemcpyAsync(Hk, hk.p, 16 * (size_t)n * nw2, cudaMemcpyDefault, c->stream));
    TRY(launch_heevj(c, n, c->nw, hk.p, nullptr, e.p, u.p));
    if (eps) PGB_CUDA_TRY(c, cudaMemcpyAsync(eps, e.p, 8 * (size_t)n * c->nw, cudaMemcpyDefault, c->stream));
    if (U) PGB_CUDA_TRY(c, cudaMemcpyAsync(U, u.p, 16 * (size_t)n * nw2, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

// shared body of pgb_diag_bands_mixed (H, nw bands) and pgb_diag_phonons_mixed (mass-scaled D, nm modes)
static pgb_status diag_mixed(pgb_ctx *c, const HermTab &tab, int nn, bool refine, const char *who, const double *pts,
                             int64_t n, double *Hp, double *eps, float *U) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_model) return fail(c, PGB_ESTATE, std::string(who) + ": call set_model first");
    if (nn < 2) return fail(c, PGB_EINVAL, std::string(who) + ": needs matrices of size >= 2");
    if (n < 0) return fail(c, PGB_EINVAL, std::string(who) + ": negative n");
    if (n == 0) return PGB_OK;
    if (!pts) return fail(c, PGB_EINVAL, std::string(who) + ": null pts");
    const int nw2 = nn * nn;
    In<double> P;
    TRY(P.init(c, pts, 3 * (size_t)n));
    Tmp<double> hp, e;
    Tmp<float2> u;
    TRY(hp.alloc(c, (size_t)n * nw2));
    TRY(e.alloc(c, (size_t)n * nn));
    TRY(u.alloc(c, (size_t)n * nw2));
    TRY(launch_herm_sum(c, tab, P.dev, n, hp.p));
    if (Hp) PGB_CUDA_TRY(c, cudaMemcpyAsync(Hp, hp.p, 8 * (size_t)n * nw2, cudaMemcpyDefault, c->stream));
    TRY(launch_heev_mixed(c, n, nn, hp.p, e.p, u.p, nullptr, refine));
    if (eps) PGB_CUDA_TRY(c, cudaMemcpyAsync(eps, e.p, 8 * (size_t)n * nn, cudaMemcpyDefault, c->stream));
    if (U) PGB_CUDA_TRY(c, cudaMemcpyAsync(U, u.p, 8 * (size_t)n * nw2, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status pgb_diag_bands_mixed(pgb_ctx *c, const double *pts, int64_t n, double *Hp, double *eps, float *U) {
    if (!c) return PGB_EINVAL;
    return diag_mixed(c, c->htH, c->nw, false, "diag_bands_mixed", pts, n, Hp, eps, U);
}

pgb_status pgb_diag_phonons_mixed(pgb_ctx *c, const double *pts, int64_t n, double *Dp, double *w2, float *e) {
    if (!c) return PGB_EINVAL;
    return diag_mixed(c, c->htD, c->nm, true, "diag_phonons_mixed", pts, n, Dp, w2, e);
}

pgb_status pgb_build_collision_grid(pgb_ctx *c, int band_lo, int band_hi, double e_lo, double e_hi, double T,
                                    double sigma, int64_t *nnz_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) return fail(c, PGB_ESTATE, "build_collision_grid: call set_grids first");
    for (int d = 0; d < 3; ++d)
        if (c->kg[d] != c->qg[d]) return fail(c, PGB_EINVAL, "build_collision_grid: the q grid must equal the k grid");
    if (band_lo < 0 || band_hi > c->nw || band_lo >= band_hi)
        return fail(c, PGB_EINVAL, "build_collision_grid: need 0 <= band_lo < band_hi <= nw");
    if (!(T > 0.0) || !(sigma > 0.0) || !(e_lo <= e_hi))
        return fail(c, PGB_EINVAL, "build_collision_grid: need T > 0, sigma > 0, e_lo <= e_hi");
    const int nbnd = band_hi - band_lo;
    const int64_t ns = c->Nk * nbnd;
    if (ns > (1 << 24)) return fail(c, PGB_EINVAL, "build_collision_grid: too many states");
    free_coll(c);
    const int nw = c->nw, nm = c->nm;
    const int64_t ncol = (int64_t)nm * nw * nw, nrow = (int64_t)c->nKp * ncol, nsub = (int64_t)nbnd * nm * nw;
    const int64_t nrowS = (int64_t)c->nRgp * ncol;
    // window flags and the k-points that hold at least one window state
    std::vector<double> eps((size_t)c->Nk * nw);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(eps.data(), c->d_eps, 8 * eps.size(), cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<uint8_t> inwin((size_t)ns, 0);
    std::vector<int32_t> active;
    for (int64_t k = 0; k < c->Nk; ++k) {
        bool any = false;
        for (int nl = 0; nl < nbnd; ++nl) {
            const double e = eps[(size_t)k * nw + band_lo + nl];
            const bool in = e >= e_lo && e <= e_hi;
            inwin[(size_t)k * nbnd + nl] = in ? 1 : 0;
            any |= in;
        }
        if (any) active.push_back((int32_t)k);
    }
    const int64_t na = (int64_t)active.size();
    Tmp<uint8_t> d_inwin;
    Tmp<int32_t> d_active;
    TRY(d_inwin.alloc(c, (size_t)ns));
    TRY(d_active.alloc(c, (size_t)std::max<int64_t>(na, 1)));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(d_inwin.p, inwin.data(), ns, cudaMemcpyHostToDevice, c->stream));
    if (na) PGB_CUDA_TRY(c, cudaMemcpyAsync(d_active.p, active.data(), 4 * na, cudaMemcpyHostToDevice, c->stream));
    Tmp<unsigned long long> counter;
    TRY(counter.alloc(c, 1));
    PGB_CUDA_TRY(c, cudaMemsetAsync(counter.p, 0, 8, c->stream));
    ListLaunch L;
    L.nb = na;
    L.kidx = d_active.p;
    L.na = na;
    L.win = d_active.p;
    L.band_lo = band_lo;
    L.nbnd = nbnd;
    L.inwin = d_inwin.p;
    L.cut = kDeltaCut * sigma;
    TRY(list_count(c, L, counter.p));
    unsigned long long total = 0;
    PGB_CUDA_TRY(c, cudaMemcpyAsync(&total, counter.p, 8, cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (total > (unsigned long long)INT32_MAX * 8)
        return fail(c, PGB_EINVAL, "build_collision_grid: list too large");
    // keys and values, with the radix sort's alternate buffers
    Tmp<uint64_t> keys, keys2;
    Tmp<float> vals, vals2;
    TRY(keys.alloc(c, (size_t)std::max<unsigned long long>(total, 1)));
    TRY(keys2.alloc(c, (size_t)std::max<unsigned long long>(total, 1)));
    TRY(vals.alloc(c, (size_t)std::max<unsigned long long>(total, 1)));
    TRY(vals2.alloc(c, (size_t)std::max<unsigned long long>(total, 1)));
    PGB_CUDA_TRY(c, cudaMemsetAsync(counter.p, 0, 8, c->stream));
    // q-grid phases (FP32, kept for later calls)
    if (!c->d_phq32) {
        TRY(dalloc(c, &c->d_phq32, (size_t)c->Nq * c->nKp));
        TRY(launch_qtable_grid(c, nullptr, c->Nq, c->d_phq32, true));
    }
    const size_t es = sizeof(float2);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // per k: R_e phases, S1, G, the gathered q rows (only q = k' - k with k' in the window) and C
    const size_t per_k = al(c->nRge * es) + 2 * al(nrow * es) + al((size_t)na * c->nKp * es) + al((size_t)na * nsub * es);
    int64_t nbmax = std::max<int64_t>(1, (int64_t)(((size_t)4 << 30) / per_k));
    nbmax = std::min<int64_t>(nbmax, std::max<int64_t>(na, 1));
    nbmax = std::min<int64_t>(nbmax, 65535);
    TRY(ensure_scratch(c, nbmax * per_k + 4096));
    char *base = (char *)c->scratch;
    char *phk = base;
    char *S1 = phk + al(nbmax * c->nRge * es);
    char *G = S1 + al(nbmax * nrow * es);
    char *phg = G + al(nbmax * nrow * es);
    char *Cb = phg + al(nbmax * na * c->nKp * es);
    for (int64_t b0 = 0; b0 < na; b0 += nbmax) {
        const int64_t nb = std::min<int64_t>(nbmax, na - b0);
        const int32_t *kb = d_active.p + b0;
        TRY(launch_phase_grid(c, c->kg, kb, nb, c->d_Rge, c->nRge, phk, true));
        TRY(launch_cgemm(c, true, 1, nb, nrowS, c->nRge, phk, c->nRge, 0, c->d_g32, nrowS, 0, S1, nrowS, 0));
        TRY(launch_fold_u(c, true, nb, kb, c->nRgp, nm, nw, S1, c->d_U32, G));
        // q-sum over the window k' only (q = k' - k) and the columns of the listed bands only
        ListLaunch Lg = L;
        Lg.nb = nb;
        Lg.kidx = kb;
        TRY(list_gather_qrows(c, Lg, c->d_phq32, phg));
        TRY(launch_cgemm(c, true, nb, na, nsub, c->nKp, phg, c->nKp, na * c->nKp,
                         (const float2 *)G + (int64_t)band_lo * nm * nw, ncol, nrow, Cb, nsub, na * nsub));
        ListLaunch Lb = L;
        Lb.nb = nb;
        Lb.kidx = kb;
        TRY(list_fill(c, Lb, Cb, counter.p, keys.p, vals.p, total));
    }
    unsigned long long filled = 0;
    PGB_CUDA_TRY(c, cudaMemcpyAsync(&filled, counter.p, 8, cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (filled != total) return fail(c, PGB_ECUDA, "build_collision_grid: count and fill passes disagree");
    TRY(dalloc(c, &c->d_coo_row, (size_t)total));
    TRY(dalloc(c, &c->d_coo_col, (size_t)total));
    TRY(dalloc(c, &c->d_coo_mode, (size_t)total));
    TRY(dalloc(c, &c->d_coo_g2, (size_t)total));
    TRY(list_sort_decode(c, (int64_t)total, (int)ns, keys.p, vals.p, keys2.p, vals2.p, c->d_coo_row, c->d_coo_col,
                         c->d_coo_mode, c->d_coo_g2));
    c->band_lo = band_lo;
    c->band_hi = band_hi;
    c->nstates = ns;
    c->nnz = (int64_t)total;
    c->coll_elo = e_lo;
    c->coll_ehi = e_hi;
    pgb_status st = launch_coll_coeffs(c, T, sigma, c->d_coo_row, c->d_coo_col, c->d_coo_mode, c->d_coo_g2,
                                       (int64_t)total, nbnd);
    if (st != PGB_OK) return st;
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->has_coll = true;
    if (nnz_out) *nnz_out = (int64_t)total;
    return PGB_OK;
}

pgb_status pgb_collision_list(pgb_ctx *c, int32_t *row, int32_t *col, int32_t *mode, float *g2) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_coll) return fail(c, PGB_ESTATE, "collision_list: call build_collision first");
    const size_t n = (size_t)c->nnz;
    if (row) PGB_CUDA_TRY(c, cudaMemcpyAsync(row, c->d_coo_row, 4 * n, cudaMemcpyDefault, c->stream));
    if (col) PGB_CUDA_TRY(c, cudaMemcpyAsync(col, c->d_coo_col, 4 * n, cudaMemcpyDefault, c->stream));
    if (mode) PGB_CUDA_TRY(c, cudaMemcpyAsync(mode, c->d_coo_mode, 4 * n, cudaMemcpyDefault, c->stream));
    if (g2) PGB_CUDA_TRY(c, cudaMemcpyAsync(g2, c->d_coo_g2, 4 * n, cudaMemcpyDefault, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

}  // extern "C"

extern "C" pgb_status pgb_diag_delta_weights(pgb_ctx *c, int64_t n, const double *en, const double *em,
                                             const double *hw, double eps_ref, double sigma, float *out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (n < 0 || !(sigma > 0.0)) return fail(c, PGB_EINVAL, "diag_delta_weights: need n >= 0, sigma > 0");
    if (n == 0) return PGB_OK;
    In<double> E1, E2, W;
    TRY(E1.init(c, en, (size_t)n));
    TRY(E2.init(c, em, (size_t)n));
    TRY(W.init(c, hw, (size_t)n));
    Out<float> O;
    TRY(O.init(c, out, 4 * (size_t)n));
    if (!O.dev) return fail(c, PGB_EINVAL, "diag_delta_weights: null output");
    TRY(diag_delta_weights(c, n, E1.dev, E2.dev, W.dev, eps_ref, sigma, O.dev));
    TRY(O.finish());
    return PGB_OK;
}

extern "C" int64_t pgb_diag_alloc_count(void) { return pgb::alloc_hook::count.load(); }

extern "C" void pgb_diag_fail_alloc(int64_t n) {
    pgb::alloc_hook::fail.store(n < 0 ? -1 : pgb::alloc_hook::count.load() + n);
}
