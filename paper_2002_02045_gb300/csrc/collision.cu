// Collision integral I[f] (Eq. e_ph_scattering) on a CSR scattering list and
// the fused RK4 stages (Sec. 2.1.1).
#include <vector>

#include "coeffs.cuh"
#include "internal.cuh"

namespace pgb {

static inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// list validation: bit 0 row out of range, 1 col out of range, 2 mode out of
// range, 3 rows decreasing, 4 band of a state outside [band_lo, band_hi)
// ---------------------------------------------------------------------------
__global__ void k_coll_validate(int64_t nnz, int64_t nstates, int nm, const int32_t *__restrict__ row,
                                const int32_t *__restrict__ col, const int32_t *__restrict__ mode,
                                int *__restrict__ flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int f = 0;
    const int32_t r = row[e];
    if (r < 0 || r >= nstates) f |= 1;
    const int32_t cc = col[e];
    if (cc < 0 || cc >= nstates) f |= 2;
    const int32_t md = mode[e];
    if (md < 0 || md >= nm) f |= 4;
    if (e > 0 && row[e - 1] > r) f |= 8;
    if (f) atomicOr(flag, f);
}

// ---------------------------------------------------------------------------
// Per-entry coefficients, FP64 arithmetic, stored FP32:
//   a = scale |g|^2 [d_em (N+1) + d_abs N],  b = scale |g|^2 [d_em N + d_abs (N+1)]
// scale = (2 pi/hbar) / (N_q s sqrt(pi)).  The reverse entry of a process gets
// a' = b and b' = a bit for bit (coll_brackets), so that sum_s I_s = 0 is not
// broken by the list.
// ---------------------------------------------------------------------------
struct CoeffArgs {
    int64_t nnz;
    const int32_t *row, *col, *mode;
    const float *g2;
    CoeffGeom g;
    int32_t *out_col;
    float *a, *b;
};

__global__ void k_coll_coeffs(CoeffArgs p) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.nnz) return;
    double ca, cb;
    coll_brackets(p.g, p.row[e], p.col[e], p.mode[e], ca, cb);
    const double gs = p.g.scale * (double)p.g2[e];
    p.out_col[e] = p.col[e];
    p.a[e] = (float)(gs * ca);
    p.b[e] = (float)(gs * cb);
}

__global__ void k_rowptr(int64_t nstates, int64_t nnz, const int32_t *__restrict__ row, int64_t *__restrict__ rowptr) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nstates) return;
    int64_t lo = 0, hi = nnz;   // first e with row[e] >= s
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row[mid] < s)
            lo = mid + 1;
        else
            hi = mid;
    }
    rowptr[s] = lo;
}

__global__ void k_eps_state(int64_t nstates, int nb, int band_lo, int nw, const double *__restrict__ eps,
                            double *__restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstates) return;
    out[s] = eps[(s / nb) * nw + (s % nb) + band_lo];
}

// warp per row: sum of a (FP64) for the -f_s sum_e a_e term
__global__ void k_rowsum(int64_t nstates, const int64_t *__restrict__ rowptr, const float *__restrict__ a,
                         double *__restrict__ out) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nstates) return;
    double acc = 0.0;
    for (int64_t e = rowptr[s] + lane; e < rowptr[s + 1]; e += 32) acc += (double)a[e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[s] = acc;
}

CoeffGeom coeff_geom(const pgb_ctx *c) {
    CoeffGeom g;
    g.nb = c->coll_nb;
    g.band_lo = c->band_lo;
    g.nw = c->nw;
    g.nm = c->nm;
    for (int d = 0; d < 3; ++d) g.kg[d] = c->kg[d];
    g.eps = c->d_eps;
    g.hw = c->d_hw;
    g.T = c->coll_T;
    g.sigma = c->coll_sigma;
    g.scale = kTwoPiOverHbar / ((double)c->Nq * c->coll_sigma * kSqrtPi);
    return g;
}

// a, b (and the column copy) of every entry from |g|^2; the row sums of a follow
// once the row pointers exist.
pgb_status launch_coll_values(pgb_ctx *c, const int32_t *row, const int32_t *col, const int32_t *mode,
                              const float *g2, int64_t nnz) {
    if (nnz == 0) return PGB_OK;
    CoeffArgs p;
    p.nnz = nnz;
    p.row = row;
    p.col = col;
    p.mode = mode;
    p.g2 = g2;
    p.g = coeff_geom(c);
    p.out_col = c->d_col;
    p.a = c->d_a;
    p.b = c->d_b;
    k_coll_coeffs<<<div_up(nnz, 256), 256, 0, c->stream>>>(p);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_coll_rowsum(pgb_ctx *c) {
    if (c->nstates == 0) return PGB_OK;
    k_rowsum<<<div_up(c->nstates * 32, 256), 256, 0, c->stream>>>(c->nstates, c->d_rowptr, c->d_a, c->d_rowsum_a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_coll_coeffs(pgb_ctx *c, double T, double sigma, const int32_t *row, const int32_t *col,
                              const int32_t *mode, const float *g2, int64_t nnz, int nb) {
    const int64_t ns = c->nstates;
    if (nnz > 0) {
        int *d_flag = nullptr;
        PGB_CUDA_TRY(c, dev_malloc_async((void **)&d_flag, sizeof(int), c->stream));
        PGB_CUDA_TRY(c, cudaMemsetAsync(d_flag, 0, sizeof(int), c->stream));
        k_coll_validate<<<div_up(nnz, 256), 256, 0, c->stream>>>(nnz, ns, c->nm, row, col, mode, d_flag);
        PGB_LAUNCH_CHECK(c);
        int flag = 0;
        PGB_CUDA_TRY(c, cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaFreeAsync(d_flag, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (flag) {
            c->err = "build_collision: invalid list (flags " + std::to_string(flag) +
                     ": 1 row range, 2 col range, 4 mode range, 8 rows not sorted)";
            return PGB_EINVAL;
        }
    }
    pgb_status st;
    if ((st = dalloc(c, &c->d_eps_state, ns)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_rowptr, ns + 1)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_col, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_a, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_b, nnz)) != PGB_OK) return st;
    if ((st = dalloc(c, &c->d_rowsum_a, ns)) != PGB_OK) return st;
    for (int i = 0; i < 3; ++i)
        if ((st = dalloc(c, &c->d_f[i], ns)) != PGB_OK) return st;
    for (int i = 0; i < 3; ++i)
        if ((st = dalloc(c, &c->d_f32[i], ns)) != PGB_OK) return st;

    k_eps_state<<<div_up(ns, 256), 256, 0, c->stream>>>(ns, nb, c->band_lo, c->nw, c->d_eps, c->d_eps_state);
    PGB_LAUNCH_CHECK(c);
    c->coll_T = T;
    c->coll_sigma = sigma;
    c->coll_nb = nb;
    if ((st = launch_coll_values(c, row, col, mode, g2, nnz)) != PGB_OK) return st;
    k_rowptr<<<div_up(ns + 1, 256), 256, 0, c->stream>>>(ns, nnz, row, c->d_rowptr);
    PGB_LAUNCH_CHECK(c);
    k_rowsum<<<div_up(ns * 32, 256), 256, 0, c->stream>>>(ns, c->d_rowptr, c->d_a, c->d_rowsum_a);
    PGB_LAUNCH_CHECK(c);
    // non-empty rows, the only ones the collision kernel visits
    std::vector<int64_t> rp((size_t)ns + 1);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(rp.data(), c->d_rowptr, 8 * rp.size(), cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> act;
    for (int64_t r = 0; r < ns; ++r)
        if (rp[r + 1] > rp[r]) act.push_back((int32_t)r);
    c->nrows_active = (int64_t)act.size();
    if ((st = dalloc(c, &c->d_active_rows, std::max<size_t>(act.size(), 1))) != PGB_OK) return st;
    if (!act.empty())
        PGB_CUDA_TRY(c, cudaMemcpyAsync(c->d_active_rows, act.data(), 4 * act.size(), cudaMemcpyHostToDevice,
                                        c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

// ---------------------------------------------------------------------------
// I_s = -f_s sum_e a_e + f_s sum_e f_c a_e + (1 - f_s) sum_e f_c b_e
// (the bracket of Eq. e_ph_scattering expanded: -f_s(1-f_c) a + f_c(1-f_s) b).
// One 256-thread block per non-empty row (rows of the dynamics workload hold
// ~2e4 entries, so a row needs many loads in flight).  Entries stream as
// 16-byte vectors (4 entries per thread per step, two steps in flight) once the
// row is 16-byte aligned.  The FP64 rate is a small fraction of the FP32 rate,
// so no per-entry work touches FP64: f_c is gathered from an FP32 copy written
// by the previous stage, products and running sums are FP32 with Kahan
// compensation, and only the per-row combination is FP64.  Stage -1 writes I; stages 0..3 fuse the RK4
// combinations (any stage can also write the diagonal of dI/df, which the
// reverse-mode pass needs):
//   0: acc = k1,  next = f + dt/2 k1      1: acc += 2 k2, next = f + dt/2 k2
//   2: acc += 2 k3, next = f + dt k3      3: f = f + dt/6 (acc + k4)
// Empty rows have I = 0 and are not launched; their stage values stay f.
// ---------------------------------------------------------------------------
struct CollArgs {
    int64_t nrows;           // non-empty rows
    const int32_t *rows;     // [nrows] state index of each non-empty row
    const int64_t *rowptr;
    const int32_t *col;
    const float *a, *b;
    const double *rowsum_a;
    const double *fin;    // occupations the integral is evaluated at
    const float *fin32;   // FP32 copy of fin (gathered per entry)
    const double *fbase;  // f at the start of the step
    double *I;            // stage -1 output
    double *acc;
    double *fnext;
    float *fnext32;       // FP32 copy of fnext (stages 0..3)
    double *D;            // if set: dI_s/df_s = -sum a + sum f_c a - sum f_c b (any stage)
    double dt;            // seconds
    int stage;
};

constexpr int kCollThreads = 256;

__global__ void __launch_bounds__(kCollThreads) k_collision(CollArgs p) {
    __shared__ double red[2][kCollThreads / 32];
    const int64_t r = blockIdx.x;
    if (r >= p.nrows) return;
    const int s = p.rows[r];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t beg = p.rowptr[s], end = p.rowptr[s + 1];
    const float *__restrict__ f32 = p.fin32;
    // Kahan-compensated FP32 sums
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    auto kadd = [](float &sum, float &comp, float x) {
        const float y = x - comp;
        const float t2 = sum + y;
        comp = (t2 - sum) - y;
        sum = t2;
    };
    int64_t vbeg = (beg + 3) & ~(int64_t)3;
    if (vbeg > end) vbeg = end;
    const int64_t vend = vbeg + ((end - vbeg) & ~(int64_t)3);
    {   // head (up to 3 entries) and tail (up to 3 entries)
        int64_t e = -1;
        if (t < vbeg - beg)
            e = beg + t;
        else if (t >= 4 && t - 4 < end - vend)
            e = vend + (t - 4);
        if (e >= 0) {
            const float fc = f32[p.col[e]];
            kadd(sa, ca, fc * p.a[e]);
            kadd(sb, cb, fc * p.b[e]);
        }
    }
    const int4 *col4 = reinterpret_cast<const int4 *>(p.col + vbeg);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.a + vbeg);
    const float4 *b4 = reinterpret_cast<const float4 *>(p.b + vbeg);
    const int64_t nv = (vend - vbeg) >> 2;
#pragma unroll 2
    for (int64_t v = t; v < nv; v += kCollThreads) {
        const int4 cc = __ldcs(col4 + v);
        const float4 aa = __ldcs(a4 + v);
        const float4 bb = __ldcs(b4 + v);
        const float f0 = __ldg(f32 + cc.x), f1 = __ldg(f32 + cc.y);
        const float f2 = __ldg(f32 + cc.z), f3 = __ldg(f32 + cc.w);
        kadd(sa, ca, fmaf(f0, aa.x, fmaf(f1, aa.y, fmaf(f2, aa.z, f3 * aa.w))));
        kadd(sb, cb, fmaf(f0, bb.x, fmaf(f1, bb.y, fmaf(f2, bb.z, f3 * bb.w))));
    }
    double sfa = (double)sa - (double)ca, sfb = (double)sb - (double)cb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sfa += __shfl_down_sync(0xffffffffu, sfa, o);
        sfb += __shfl_down_sync(0xffffffffu, sfb, o);
    }
    if (lane == 0) {
        red[0][warp] = sfa;
        red[1][warp] = sfb;
    }
    __syncthreads();
    if (t == 0) {
        sfa = 0.0;
        sfb = 0.0;
        for (int w = 0; w < kCollThreads / 32; ++w) {
            sfa += red[0][w];
            sfb += red[1][w];
        }
        const double fs = p.fin[s];
        const double I = -fs * p.rowsum_a[s] + fs * sfa + (1.0 - fs) * sfb;
        if (p.D) p.D[s] = -p.rowsum_a[s] + sfa - sfb;
        double fn = 0.0;
        switch (p.stage) {
            case -1:
                p.I[s] = I;
                break;
            case 0:
                p.acc[s] = I;
                fn = p.fbase[s] + 0.5 * p.dt * I;
                break;
            case 1:
                p.acc[s] += 2.0 * I;
                fn = p.fbase[s] + 0.5 * p.dt * I;
                break;
            case 2:
                p.acc[s] += 2.0 * I;
                fn = p.fbase[s] + p.dt * I;
                break;
            default:
                fn = p.fbase[s] + p.dt / 6.0 * (p.acc[s] + I);
                break;
        }
        if (p.stage >= 0) {
            p.fnext[s] = fn;
            p.fnext32[s] = (float)fn;
        }
    }
}

__global__ void k_to_f32_real(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) y[t] = (float)x[t];
}

pgb_status launch_f64_to_f32(pgb_ctx *c, const double *x, float *y, int64_t n) {
    if (n == 0) return PGB_OK;
    k_to_f32_real<<<div_up(n, 256), 256, 0, c->stream>>>(x, y, n);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_collision(pgb_ctx *c, const double *f, const float *f32, double *I, int stage, double dt,
                            double *acc, double *fnext, float *fnext32, const double *fbase, double *D) {
    if (c->nstates == 0) return PGB_OK;
    if (stage == -1) PGB_CUDA_TRY(c, cudaMemsetAsync(I, 0, 8 * (size_t)c->nstates, c->stream));
    if (c->nrows_active == 0) return PGB_OK;
    CollArgs p;
    p.nrows = c->nrows_active;
    p.rows = c->d_active_rows;
    p.rowptr = c->d_rowptr;
    p.col = c->d_col;
    p.a = c->d_a;
    p.b = c->d_b;
    p.rowsum_a = c->d_rowsum_a;
    p.fin = f;
    p.fin32 = f32;
    p.fbase = fbase;
    p.I = I;
    p.acc = acc;
    p.fnext = fnext;
    p.fnext32 = fnext32;
    p.D = D;
    p.dt = dt;
    p.stage = stage;
    prof_mark(c, PGB_PROF_COLLISION);
    k_collision<<<(unsigned)c->nrows_active, kCollThreads, 0, c->stream>>>(p);
    prof_mark(c, PGB_PROF_COLLISION);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb
