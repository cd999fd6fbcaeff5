// Reverse-mode derivatives of the collision integral (Eq. e_ph_scattering) and
// of the RK4 time stepping (Sec. 2.1.1): gradients of a loss on f(t_end) with
// respect to f(0) and to |g|^2 of every list entry.
//
// With I_s(x) = -x_s SA_s + x_s SFA_s + (1 - x_s) SFB_s (sums over the entries
// of row s: SA = sum a, SFA = sum x_c a, SFB = sum x_c b),
//   (J^T k)_c = k_c D_c + sum_{e: col(e) = c} [u_r a_e + w_r b_e],  r = row(e),
//   D_c = -SA_c + SFA_c - SFB_c,  u_r = k_r x_r,  w_r = k_r (1 - x_r),
// and, since a_e = |g|^2_e alpha_e and b_e = |g|^2_e beta_e,
//   sum_s k_s dI_s/d|g|^2_e = w_r x_c beta_e - u_r (1 - x_c) alpha_e.
// D comes out of the forward stage kernel.  The column sums run over a
// transposed copy of the list (entries ordered by column, built once per
// list), one block per non-empty column, with the forward kernel's arithmetic:
// 16-byte entry vectors, FP32 gathers and products with Kahan sums, FP64 per
// column.  The per-entry |g|^2 derivative accumulates over all stages and
// steps in a Kahan-compensated FP32 pair (8 bytes, no FP64 arithmetic per
// entry: GB300's FP64 rate would otherwise bound the pass).
//
// RK4 reverse step (x1 = f, x2 = f + dt/2 k1, x3 = f + dt/2 k2, x4 = f + dt k3,
// f' = f + dt/6 (k1 + 2 k2 + 2 k3 + k4)) for lam = dL/df':
//   v4 = J(x4)^T (dt/6 lam)
//   v3 = J(x3)^T (dt/3 lam + dt v4)
//   v2 = J(x2)^T (dt/3 lam + dt/2 v3)
//   v1 = J(x1)^T (dt/6 lam + dt/2 v2)
//   dL/df = lam + v1 + v2 + v3 + v4
// The forward pass keeps f every `ckpt` steps and runs the last segment with
// the stage kernels storing every stage state and D.  The reverse pass
// recomputes each earlier segment the same way from its checkpoint (the
// recomputed states are bit-identical to the forward ones), and each reverse
// step is four column passes.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cub/device/device_radix_sort.cuh>

#include "coeffs.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }
constexpr int kThreads = 256;

__device__ __forceinline__ void kadd(float &s, float &comp, float v) {
    const float y = v - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
}

// ---------------------------------------------------------------------------
// transposed list
// ---------------------------------------------------------------------------
__global__ void k_iota(int64_t n, int32_t *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (int32_t)t;
}

struct GatherArgs {
    int64_t nnz;
    const int32_t *eidx;   // sorted by column
    const int32_t *row, *col, *mode;
    const float *a, *b;
    CoeffGeom g;
    int32_t *src;
    float *ta, *tb, *alpha, *beta;
};

__global__ void k_t_gather(GatherArgs p) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.nnz) return;
    const int32_t e = p.eidx[j];
    const int32_t r = p.row[e];
    double ca, cb;
    coll_brackets(p.g, r, p.col[e], p.mode[e], ca, cb);
    p.src[j] = r;
    p.ta[j] = p.a[e];
    p.tb[j] = p.b[e];
    p.alpha[j] = (float)(p.g.scale * ca);
    p.beta[j] = (float)(p.g.scale * cb);
}

__global__ void k_colptr(int64_t nstates, int64_t nnz, const int32_t *__restrict__ scol, int64_t *__restrict__ ptr) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nstates) return;
    int64_t lo = 0, hi = nnz;   // first j with scol[j] >= s
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (scol[mid] < s)
            lo = mid + 1;
        else
            hi = mid;
    }
    ptr[s] = lo;
}

// ---------------------------------------------------------------------------
// reverse-pass kernels
// ---------------------------------------------------------------------------
// k = cl*lam + cv*vprev; smode 1: sumv = vprev, 2: sumv += vprev;
// uw = (k x, k (1 - x)) in FP32 for the gathers; vout = k D (the diagonal part).
__global__ void k_adj_prep(int64_t n, const double *__restrict__ lam, double cl, const double *__restrict__ vprev,
                           double cv, const double *__restrict__ x, const double *__restrict__ D,
                           double *__restrict__ sumv, int smode, float2 *__restrict__ uw, double *__restrict__ vout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double vp = vprev ? vprev[t] : 0.0;
    const double k = cl * lam[t] + cv * vp;
    if (smode == 1)
        sumv[t] = vp;
    else if (smode == 2)
        sumv[t] += vp;
    const double xs = x[t];
    uw[t] = make_float2((float)(k * xs), (float)(k * (1.0 - xs)));
    vout[t] = k * D[t];
}

__global__ void k_adj_finish(int64_t n, double *__restrict__ lam, const double *__restrict__ sumv,
                             const double *__restrict__ v1) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) lam[t] += sumv[t] + v1[t];
}

__global__ void k_scatter_dg2(int64_t nnz, const int32_t *__restrict__ eidx, const float2 *__restrict__ acc,
                              double *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nnz) out[eidx[j]] = (double)acc[j].x - (double)acc[j].y;
}

// copies of one state into `count` consecutive state slots
__global__ void k_bcast(int64_t n, int64_t count, const double *__restrict__ src, double *__restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * count) return;
    dst[t] = src[t % n];
}

struct ColArgs {
    int64_t ncols;
    const int32_t *cols;      // non-empty columns
    const int64_t *colptr;
    const int32_t *src;
    const float *a, *b, *alpha, *beta;
    const float2 *uw;
    const double *x;
    double *v;                // v[c] += sum over the column
    float2 *acc;              // [nnz] |g|^2 derivative, transposed order, as (sum, compensation) (null: skipped)
};

__global__ void __launch_bounds__(kThreads, 5) k_adj_col(ColArgs p) {
    __shared__ double red[kThreads / 32];
    const int64_t r = blockIdx.x;
    if (r >= p.ncols) return;
    const int c = p.cols[r];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t beg = p.colptr[c], end = p.colptr[c + 1];
    const float xc = (float)p.x[c], omx = (float)(1.0 - p.x[c]);
    float s = 0.f, cs = 0.f;
    int64_t vbeg = (beg + 3) & ~(int64_t)3;
    if (vbeg > end) vbeg = end;
    const int64_t vend = vbeg + ((end - vbeg) & ~(int64_t)3);
    {   // head (up to 3 entries) and tail (up to 3 entries)
        int64_t j = -1;
        if (t < vbeg - beg)
            j = beg + t;
        else if (t >= 4 && t - 4 < end - vend)
            j = vend + (t - 4);
        if (j >= 0) {
            const float2 q = p.uw[p.src[j]];
            kadd(s, cs, fmaf(q.x, p.a[j], q.y * p.b[j]));
            if (p.acc) {
                float2 d = p.acc[j];
                kadd(d.x, d.y, q.y * xc * p.beta[j] - q.x * omx * p.alpha[j]);
                p.acc[j] = d;
            }
        }
    }
    const int64_t nv = (vend - vbeg) >> 2;
#pragma unroll 2
    for (int64_t v = t; v < nv; v += kThreads) {
        const int64_t j = vbeg + 4 * v;
        const int4 sr = __ldcs(reinterpret_cast<const int4 *>(p.src + j));
        const float4 aa = __ldcs(reinterpret_cast<const float4 *>(p.a + j));
        const float4 bb = __ldcs(reinterpret_cast<const float4 *>(p.b + j));
        const float2 q0 = __ldg(p.uw + sr.x), q1 = __ldg(p.uw + sr.y);
        const float2 q2 = __ldg(p.uw + sr.z), q3 = __ldg(p.uw + sr.w);
        kadd(s, cs, fmaf(q0.x, aa.x, fmaf(q0.y, bb.x, fmaf(q1.x, aa.y, q1.y * bb.y))));
        kadd(s, cs, fmaf(q2.x, aa.z, fmaf(q2.y, bb.z, fmaf(q3.x, aa.w, q3.y * bb.w))));
        if (p.acc) {
            const float4 al = __ldcs(reinterpret_cast<const float4 *>(p.alpha + j));
            const float4 be = __ldcs(reinterpret_cast<const float4 *>(p.beta + j));
            // Kahan-compensated FP32 pairs: no FP64 arithmetic per entry
            float4 *ap = reinterpret_cast<float4 *>(p.acc + j);
            float4 lo = ap[0], hi = ap[1];   // (sum, comp) of entries j, j+1 and j+2, j+3
            kadd(lo.x, lo.y, q0.y * xc * be.x - q0.x * omx * al.x);
            kadd(lo.z, lo.w, q1.y * xc * be.y - q1.x * omx * al.y);
            kadd(hi.x, hi.y, q2.y * xc * be.z - q2.x * omx * al.z);
            kadd(hi.z, hi.w, q3.y * xc * be.w - q3.x * omx * al.w);
            ap[0] = lo;
            ap[1] = hi;
        }
    }
    double sum = (double)s - (double)cs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) red[warp] = sum;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
        p.v[c] += tot;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Device buffers of one call, released together (stream-ordered).
struct Pool {
    pgb_ctx *c;
    std::vector<void *> ptrs;
    bool ok = true;
    explicit Pool(pgb_ctx *ctx) : c(ctx) {}
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (dev_malloc_async(&p, std::max<size_t>(count * sizeof(T), 16), c->stream) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Pool() {
        for (void *p : ptrs) cudaFreeAsync(p, c->stream);
    }
};

pgb_status launch_t_gather(pgb_ctx *c) {
    GatherArgs g;
    g.nnz = c->nnz;
    g.eidx = c->d_t_eidx;
    g.row = c->d_coo_row;
    g.col = c->d_coo_col;
    g.mode = c->d_coo_mode;
    g.a = c->d_a;
    g.b = c->d_b;
    g.g = coeff_geom(c);
    g.src = c->d_t_src;
    g.ta = c->d_t_a;
    g.tb = c->d_t_b;
    g.alpha = c->d_t_alpha;
    g.beta = c->d_t_beta;
    k_t_gather<<<div_up(c->nnz, 256), 256, 0, c->stream>>>(g);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status adj_prepare(pgb_ctx *c) {
    if (c->adj_ready) return PGB_OK;
    const int64_t ns = c->nstates, nnz = c->nnz;
    if (nnz >= ((int64_t)1 << 31)) {
        c->err = "adjoint: lists of 2^31 or more entries are not supported";
        return PGB_EINVAL;
    }
    pgb_status st;
    if ((st = dalloc(c, &c->d_t_colptr, ns + 1)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_src, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_eidx, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_a, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_b, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_alpha, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_t_beta, nnz)) != PGB_OK) return st;
    if (nnz == 0) {
        PGB_CUDA_TRY(c, cudaMemsetAsync(c->d_t_colptr, 0, 8 * (size_t)(ns + 1), c->stream));
    } else {
        Pool pool(c);
        int32_t *keys = pool.get<int32_t>(nnz), *keys2 = pool.get<int32_t>(nnz);
        int32_t *vals2 = pool.get<int32_t>(nnz);
        if (!pool.ok) {
            c->err = "adjoint: device allocation failed";
            return PGB_ENOMEM;
        }
        PGB_CUDA_TRY(c, cudaMemcpyAsync(keys, c->d_coo_col, 4 * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
        k_iota<<<div_up(nnz, 256), 256, 0, c->stream>>>(nnz, c->d_t_eidx);
        PGB_LAUNCH_CHECK(c);
        int end_bit = 1;
        while (end_bit < 31 && (1ll << end_bit) < ns) ++end_bit;
        // stable: entries of one column stay in list (row) order
        cub::DoubleBuffer<int32_t> dk(keys, keys2), dv(c->d_t_eidx, vals2);
        size_t tmp_bytes = 0;
        PGB_CUDA_TRY(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, dk, dv, nnz, 0, end_bit, c->stream));
        void *tmp = pool.get<char>(tmp_bytes);
        if (!tmp) {
            c->err = "adjoint: device allocation failed";
            return PGB_ENOMEM;
        }
        PGB_CUDA_TRY(c, cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, dk, dv, nnz, 0, end_bit, c->stream));
        c->launches += 1;
        if (dv.Current() != c->d_t_eidx)
            PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_t_eidx, dv.Current(), 4 * (size_t)nnz, cudaMemcpyDeviceToDevice,
                                            c->stream));
        if ((st = launch_t_gather(c)) != PGB_OK) return st;
        k_colptr<<<div_up(ns + 1, 256), 256, 0, c->stream>>>(ns, nnz, dk.Current(), c->d_t_colptr);
        PGB_LAUNCH_CHECK(c);
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    std::vector<int64_t> cp((size_t)ns + 1);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(cp.data(), c->d_t_colptr, 8 * cp.size(), cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> act;
    for (int64_t s = 0; s < ns; ++s)
        if (cp[s + 1] > cp[s]) act.push_back((int32_t)s);
    c->t_nactive = (int64_t)act.size();
    if ((st = dalloc(c, &c->d_t_active, std::max<size_t>(act.size(), 1))) != PGB_OK) return st;
    if (!act.empty())
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_t_active, act.data(), 4 * act.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->adj_ready = true;
    return PGB_OK;
}

struct Rev {
    pgb_ctx *c;
    int64_t ns;
    float2 *uw;
    double *sumv, *v[2];
    float2 *acc;   // null: no |g|^2 derivative
};

pgb_status prep(Rev &R, const double *lam, double cl, const double *vprev, double cv, const double *x, const double *D,
                int smode, double *vout) {
    k_adj_prep<<<div_up(R.ns, 256), 256, 0, R.c->stream>>>(R.ns, lam, cl, vprev, cv, x, D, R.sumv, smode, R.uw, vout);
    PGB_LAUNCH_CHECK(R.c);
    return PGB_OK;
}

pgb_status colpass(Rev &R, const double *x, double *v) {
    pgb_ctx *c = R.c;
    if (c->t_nactive == 0) return PGB_OK;
    ColArgs p;
    p.ncols = c->t_nactive;
    p.cols = c->d_t_active;
    p.colptr = c->d_t_colptr;
    p.src = c->d_t_src;
    p.a = c->d_t_a;
    p.b = c->d_t_b;
    p.alpha = c->d_t_alpha;
    p.beta = c->d_t_beta;
    p.uw = R.uw;
    p.x = x;
    p.v = v;
    p.acc = R.acc;
    prof_mark(c, PGB_PROF_ADJOINT);
    k_adj_col<<<(unsigned)c->t_nactive, kThreads, 0, c->stream>>>(p);
    prof_mark(c, PGB_PROF_ADJOINT);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace

void free_adjoint(pgb_ctx *c) {
    dfree(&c->d_t_colptr);
    dfree(&c->d_t_src);
    dfree(&c->d_t_eidx);
    dfree(&c->d_t_a);
    dfree(&c->d_t_b);
    dfree(&c->d_t_alpha);
    dfree(&c->d_t_beta);
    dfree(&c->d_t_active);
    c->t_nactive = 0;
    c->adj_ready = false;
}

pgb_status adjoint_values_changed(pgb_ctx *c) {
    if (!c->adj_ready || c->nnz == 0) return PGB_OK;
    return launch_t_gather(c);
}

pgb_status collision_vjp(pgb_ctx *c, const double *f, const double *lam, double *out_f, double *out_g2) {
    const int64_t ns = c->nstates, nnz = c->nnz;
    pgb_status st;
    if ((st = adj_prepare(c)) != PGB_OK) return st;
    if (ns == 0) return PGB_OK;
    Pool pool(c);
    double *D = pool.get<double>(ns), *I = pool.get<double>(ns);
    Rev R;
    R.c = c;
    R.ns = ns;
    R.uw = pool.get<float2>(ns);
    R.sumv = nullptr;
    R.v[0] = R.v[1] = nullptr;
    R.acc = out_g2 ? pool.get<float2>(nnz) : nullptr;
    if (!pool.ok) {
        c->err = "collision_vjp: device allocation failed";
        return PGB_ENOMEM;
    }
    PGB_CUDA_TRY(c, cudaMemsetAsync(D, 0, 8 * (size_t)ns, c->stream));
    if (R.acc) PGB_CUDA_TRY(c, cudaMemsetAsync(R.acc, 0, 8 * (size_t)nnz, c->stream));
    if ((st = launch_f64_to_f32(c, f, c->d_f32[0], ns)) != PGB_OK) return st;
    if ((st = launch_collision(c, f, c->d_f32[0], I, -1, 0.0, nullptr, nullptr, nullptr, nullptr, D)) != PGB_OK)
        return st;
    if ((st = prep(R, lam, 1.0, nullptr, 0.0, f, D, 0, out_f)) != PGB_OK) return st;
    if ((st = colpass(R, f, out_f)) != PGB_OK) return st;
    if (out_g2 && nnz > 0) {
        k_scatter_dg2<<<div_up(nnz, 256), 256, 0, c->stream>>>(nnz, c->d_t_eidx, R.acc, out_g2);
        PGB_LAUNCH_CHECK(c);
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

pgb_status rk4_adjoint(pgb_ctx *c, const double *f0, double dt_fs, int64_t nsteps, int64_t ckpt,
                       const double *lam_end, double *lam0, double *dg2, double *f_end) {
    const int64_t ns = c->nstates, nnz = c->nnz;
    const size_t nb8 = 8 * (size_t)ns, nb4 = 4 * (size_t)ns;
    const double dt = dt_fs * kFemto;
    pgb_status st;
    if ((st = adj_prepare(c)) != PGB_OK) return st;
    if (ckpt < 1) ckpt = 1;
    if (ckpt > nsteps) ckpt = std::max<int64_t>(nsteps, 1);
    const int64_t nseg = (nsteps + ckpt - 1) / ckpt;
    if (ns == 0) return PGB_OK;

    Pool pool(c);
    double *cps = pool.get<double>((size_t)(nseg + 1) * ns);
    double *X = pool.get<double>((size_t)4 * ckpt * ns);   // [step][stage][state]
    double *Dm = pool.get<double>((size_t)4 * ckpt * ns);
    double *cur = pool.get<double>(ns), *f1 = pool.get<double>(ns), *f2 = pool.get<double>(ns);
    double *acc4 = pool.get<double>(ns), *tail = pool.get<double>(ns);
    float *g[3] = {pool.get<float>(ns), pool.get<float>(ns), pool.get<float>(ns)};
    double *lam = pool.get<double>(ns);
    Rev R;
    R.c = c;
    R.ns = ns;
    R.uw = pool.get<float2>(ns);
    R.sumv = pool.get<double>(ns);
    R.v[0] = pool.get<double>(ns);
    R.v[1] = pool.get<double>(ns);
    R.acc = dg2 ? pool.get<float2>(nnz) : nullptr;
    if (!pool.ok) {
        c->err = "rk4_adjoint: device allocation failed";
        return PGB_ENOMEM;
    }
    if (R.acc) PGB_CUDA_TRY(c, cudaMemsetAsync(R.acc, 0, 8 * (size_t)nnz, c->stream));

    auto xs = [&](int64_t j, int i) { return X + (4 * j + i) * ns; };
    auto ds = [&](int64_t j, int i) { return Dm + (4 * j + i) * ns; };
    // n_in steps from xs(0, 0) (FP32 copy in g[0]) storing every stage state and
    // D; the state after the last step goes to `tail`
    auto stored_segment = [&](int64_t n_in) -> pgb_status {
        pgb_status s2;
        for (int64_t j = 0; j < n_in; ++j) {
            double *x0 = xs(j, 0), *nxt = j + 1 < n_in ? xs(j + 1, 0) : tail;
            if ((s2 = launch_collision(c, x0, g[0], nullptr, 0, dt, acc4, xs(j, 1), g[1], x0, ds(j, 0))) != PGB_OK)
                return s2;
            if ((s2 = launch_collision(c, xs(j, 1), g[1], nullptr, 1, dt, acc4, xs(j, 2), g[2], x0, ds(j, 1))) !=
                PGB_OK)
                return s2;
            if ((s2 = launch_collision(c, xs(j, 2), g[2], nullptr, 2, dt, acc4, xs(j, 3), g[1], x0, ds(j, 2))) !=
                PGB_OK)
                return s2;
            if ((s2 = launch_collision(c, xs(j, 3), g[1], nullptr, 3, dt, acc4, nxt, g[0], x0, ds(j, 3))) != PGB_OK)
                return s2;
        }
        return PGB_OK;
    };

    // States without entries keep f0 in every buffer and slot (their I is 0), D = 0.
    k_bcast<<<div_up(4 * ckpt * ns, 256), 256, 0, c->stream>>>(ns, 4 * ckpt, f0, X);
    PGB_LAUNCH_CHECK(c);
    PGB_CUDA_TRY(c, cudaMemsetAsync(Dm, 0, 4 * (size_t)ckpt * nb8, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(tail, f0, nb8, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(cps, f0, nb8, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(cur, f0, nb8, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(f1, f0, nb8, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(f2, f0, nb8, cudaMemcpyDeviceToDevice, c->stream));
    if ((st = launch_f64_to_f32(c, f0, g[0], ns)) != PGB_OK) return st;
    PGB_CUDA_TRY(c, cudaMemcpyAsync(g[1], g[0], nb4, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(g[2], g[0], nb4, cudaMemcpyDeviceToDevice, c->stream));
    // forward pass with the stage kernels of pgb_step_rk4, keeping f at the
    // start of every segment; the last segment, the first to be reversed,
    // stores its stage states directly
    for (int64_t sg = 0; sg < nseg; ++sg) {
        const int64_t n_in = std::min<int64_t>(ckpt, nsteps - sg * ckpt);
        if (sg == nseg - 1) {
            PGB_CUDA_TRY(c, cudaMemcpyAsync(xs(0, 0), cur, nb8, cudaMemcpyDeviceToDevice, c->stream));
            if ((st = stored_segment(n_in)) != PGB_OK) return st;
            PGB_CUDA_TRY(c, cudaMemcpyAsync(cps + (sg + 1) * ns, tail, nb8, cudaMemcpyDeviceToDevice, c->stream));
            break;
        }
        for (int64_t j = 0; j < n_in; ++j) {
            if ((st = launch_collision(c, cur, g[0], nullptr, 0, dt, acc4, f1, g[1], cur)) != PGB_OK) return st;
            if ((st = launch_collision(c, f1, g[1], nullptr, 1, dt, acc4, f2, g[2], cur)) != PGB_OK) return st;
            if ((st = launch_collision(c, f2, g[2], nullptr, 2, dt, acc4, f1, g[1], cur)) != PGB_OK) return st;
            if ((st = launch_collision(c, f1, g[1], nullptr, 3, dt, acc4, cur, g[0], cur)) != PGB_OK) return st;
        }
        PGB_CUDA_TRY(c, cudaMemcpyAsync(cps + (sg + 1) * ns, cur, nb8, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (f_end) PGB_CUDA_TRY(c, cudaMemcpyAsync(f_end, cps + nseg * ns, nb8, cudaMemcpyDeviceToDevice, c->stream));

    PGB_CUDA_TRY(c, cudaMemcpyAsync(lam, lam_end, nb8, cudaMemcpyDeviceToDevice, c->stream));
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t n_in = std::min<int64_t>(ckpt, nsteps - sg * ckpt);
        if (sg < nseg - 1) {   // recompute the segment from its checkpoint
            PGB_CUDA_TRY(c, cudaMemcpyAsync(xs(0, 0), cps + sg * ns, nb8, cudaMemcpyDeviceToDevice, c->stream));
            if ((st = launch_f64_to_f32(c, xs(0, 0), g[0], ns)) != PGB_OK) return st;
            if ((st = stored_segment(n_in)) != PGB_OK) return st;
        }
        // reverse steps
        for (int64_t j = n_in - 1; j >= 0; --j) {
            if ((st = prep(R, lam, dt / 6.0, nullptr, 0.0, xs(j, 3), ds(j, 3), 0, R.v[0])) != PGB_OK) return st;
            if ((st = colpass(R, xs(j, 3), R.v[0])) != PGB_OK) return st;                  // v4
            if ((st = prep(R, lam, dt / 3.0, R.v[0], dt, xs(j, 2), ds(j, 2), 1, R.v[1])) != PGB_OK) return st;
            if ((st = colpass(R, xs(j, 2), R.v[1])) != PGB_OK) return st;                  // v3
            if ((st = prep(R, lam, dt / 3.0, R.v[1], 0.5 * dt, xs(j, 1), ds(j, 1), 2, R.v[0])) != PGB_OK) return st;
            if ((st = colpass(R, xs(j, 1), R.v[0])) != PGB_OK) return st;                  // v2
            if ((st = prep(R, lam, dt / 6.0, R.v[0], 0.5 * dt, xs(j, 0), ds(j, 0), 2, R.v[1])) != PGB_OK) return st;
            if ((st = colpass(R, xs(j, 0), R.v[1])) != PGB_OK) return st;                  // v1
            k_adj_finish<<<div_up(ns, 256), 256, 0, c->stream>>>(ns, lam, R.sumv, R.v[1]);
            PGB_LAUNCH_CHECK(c);
        }
    }
    PGB_CUDA_TRY(c, cudaMemcpyAsync(lam0, lam, nb8, cudaMemcpyDeviceToDevice, c->stream));
    if (dg2 && nnz > 0) {
        k_scatter_dg2<<<div_up(nnz, 256), 256, 0, c->stream>>>(nnz, c->d_t_eidx, R.acc, dg2);
        PGB_LAUNCH_CHECK(c);
    }
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

}  // namespace pgb
