// Scattering rates (Eqs. scatter_rate, BTE_W) of many independent model
// instances of uneven band, mode and grid sizes in one persistent launch.
//
// Each member context holds its own model and grids.  Per call, the per-
// instance set-up (occupation tables and the R_e sums with U(k) folded) and
// one persistent kernel over the work units of every instance are captured in
// a CUDA graph, which later calls with the same arguments replay.
//
// Work unit = (instance, k, initial band n, tile of QT q-points).  A unit
//   1. forms its R_p-sum tile C[q][ka][i] = sum_p e^{iq.R_p} G_k[p][n][ka][i] in shared
//      memory, K-chunk by K-chunk (the next chunk copied by cp.async while the
//      current one is multiplied), from the instance's FP32 q table (exact grid
//      phases and, for polar models, the long-range columns; built once per
//      plan) and the G_k rows of band n, which are contiguous (column order n, ka, i);
//      in a split precision (BF16x3 / TF32x3) the non-polar instances' R_p sums
//      come from the tensor cores instead (k_tc_qsum on split operands, inside
//      the same graph, columns padded to a multiple of 96) and the unit copies
//      its band's columns of that result;
//   2. runs the rates epilogue on the tile: screen every (q, nu) against the
//      (m) with |x| <= 7 sigma, list the live pairs in order, then one live pair
//      per thread: project on nu, rotate by U(k+q) (FP32 products), then the
//      energy differences, Gaussian weights and occupation factors in FP64;
//   3. writes the sum of its terms to its own partial slot.
// Units are assigned to the persistent CTAs round-robin (every instance's
// units are spread over all CTAs); a second kernel adds the q-tile partials of
// each (instance, k, n) in order, so results do not depend on the schedule.
//
// The tile height QT and the block size are chosen by a small autotuner: on
// the first call every candidate runs once, timed with events, and the fastest
// is kept for the batch.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "cplx.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }
constexpr int KC = 8;    // K chunk of the shared-memory GEMM (double-buffered)
constexpr int RT = 4;    // tile rows per thread in the shared-memory GEMM

struct BInst {
    int nw, nm, nRgp, nKp;
    int qg[3], kg[3];
    int64_t Nq;
    int64_t unit0;             // first unit of this instance
    int nqt;                   // q tiles
    const float2 *phq;         // [Nq][nKp] q table: e^{iq.R_p}, then the long-range columns
    const float2 *Ctc;         // [nk][Nq][ldc] q-sum from the tensor cores, or null (SIMT GEMM here)
    int ldc;                   // nm*nw*nw rounded up to a multiple of 96
    const float2 *G;           // [nk][nKp][nm*nw*nw]
    const int32_t *kidx;       // [nk]
    const double *eps;         // [Nk][nw]
    const float *eps32;        // [Nk][nw] FP32 copy for the screen
    const float *hw32;         // [Nq][nm] FP32 copy for the screen
    const float2 *U;           // [Nk][nw][nw] transposed: U[k][m][i] = U_im(k) (row m contiguous)
    const float2 *coef;        // [Nq][nm][nm]
    const double *hw;          // [Nq][nm]
    const double *focc;        // [Nk][nw]
    const double *nbe;         // [Nq][nm]
    double sigma;
};

struct BArgs {
    int ninst;
    const BInst *inst;
    const int32_t *unit_inst;  // [nunits] instance of each unit
    int64_t nunits;
    int maxc;                  // max nm*nw over the instances (shared tile width)
    double *partial;           // [nunits]
};

__device__ __forceinline__ int64_t kq_index(int64_t k, int64_t q, const int kg[3], const int qg[3]) {
    const int k3 = (int)(k % kg[2]), k2 = (int)((k / kg[2]) % kg[1]), k1 = (int)(k / ((int64_t)kg[1] * kg[2]));
    const int q3 = (int)(q % qg[2]), q2 = (int)((q / qg[2]) % qg[1]), q1 = (int)(q / ((int64_t)qg[1] * qg[2]));
    const int s1 = (k1 + q1 * (kg[0] / qg[0])) % kg[0];
    const int s2 = (k2 + q2 * (kg[1] / qg[1])) % kg[1];
    const int s3 = (k3 + q3 * (kg[2] / qg[2])) % kg[2];
    return ((int64_t)s1 * kg[1] + s2) * kg[2] + s3;
}

// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (src not read)
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int QT, int NT>
__global__ void __launch_bounds__(NT) k_batch_rates(BArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    float2 *Cs = sm;                         // [QT][maxc]
    float2 *As = Cs + QT * a.maxc;           // [2][QT][KC]
    float2 *Bs = As + 2 * QT * KC;           // [2][KC][maxc]
    __shared__ double red[NT / 32];
    __shared__ int wcnt[NT / 32];
    __shared__ int kqrow[QT];                    // k+q grid index of each tile row
    __shared__ uint32_t items[QT * kMaxNmode];   // live (q, nu) of the tile: item << 16 | mask of m
    const int t = threadIdx.x;
    for (int64_t u = blockIdx.x; u < a.nunits; u += gridDim.x) {
        const BInst I = a.inst[a.unit_inst[u]];
        const int nw = I.nw, nm = I.nm, ncn = nm * nw, ncol = nm * nw * nw;
        const int64_t r = u - I.unit0;
        const int qt = (int)(r % I.nqt);
        const int n = (int)((r / I.nqt) % nw);
        const int64_t kb = r / ((int64_t)I.nqt * nw);
        const int64_t q0 = (int64_t)qt * QT;
        const int nq = (int)(I.Nq - q0 < QT ? I.Nq - q0 : QT);
        const float2 *Gk = I.G + kb * (int64_t)I.nKp * ncol + (int64_t)n * ncn;
        if (I.Ctc) {
            // 1'. the R_p sum came from the tensor cores: copy band n's columns of the tile
            const float2 *src = I.Ctc + (kb * I.Nq + q0) * I.ldc + (int64_t)n * ncn;
            for (int o = t; o < nq * ncn; o += NT) {
                const int qq = o / ncn, cc = o - (o / ncn) * ncn;
                Cs[qq * a.maxc + cc] = src[(int64_t)qq * I.ldc + cc];
            }
            __syncthreads();
        }
        for (int o = t; o < QT * ncn && !I.Ctc; o += NT) Cs[(o / ncn) * a.maxc + o % ncn] = make_float2(0.f, 0.f);
        // 1. R_p-sum tile; K chunk c + 1 is copied (cp.async) while chunk c is multiplied
        const int nch = I.Ctc ? 0 : (I.nKp + KC - 1) / KC;
        auto fill = [&](int c) {
            const int p0 = c * KC;
            float2 *Ab = As + (c & 1) * QT * KC, *Bb = Bs + (c & 1) * KC * a.maxc;
            for (int o = t; o < QT * KC; o += NT) {
                const int qq = o / KC, kk = o % KC;
                const bool ok = qq < nq && p0 + kk < I.nKp;
                cp_async8(Ab + o, ok ? I.phq + (q0 + qq) * I.nKp + p0 + kk : I.phq, ok ? 8 : 0);
            }
            for (int o = t; o < KC * ncn; o += NT) {
                const int kk = o / ncn, cc = o - (o / ncn) * ncn;
                const bool ok = p0 + kk < I.nKp;
                cp_async8(Bb + kk * a.maxc + cc, ok ? Gk + (int64_t)(p0 + kk) * ncol + cc : Gk, ok ? 8 : 0);
            }
            cp_async_commit();
        };
        if (nch > 0) fill(0);
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) {
                fill(c + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float2 *Ab = As + (c & 1) * QT * KC, *Bb = Bs + (c & 1) * KC * a.maxc;
            // each thread: one column, RT rows spaced QT/RT apart (one B load feeds RT products)
            for (int o = t; o < (QT / RT) * ncn; o += NT) {
                const int q0r = o / ncn, cc = o - (o / ncn) * ncn;
                float2 acc[RT];
#pragma unroll
                for (int j = 0; j < RT; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < KC; kk += 2) {
                    const float2 b0 = Bb[kk * a.maxc + cc], b1 = Bb[(kk + 1) * a.maxc + cc];
#pragma unroll
                    for (int j = 0; j < RT; ++j) {
                        const float4 av = *reinterpret_cast<const float4 *>(Ab + (q0r + j * (QT / RT)) * KC + kk);
                        cfma(acc[j], make_float2(av.x, av.y), b0);
                        cfma(acc[j], make_float2(av.z, av.w), b1);
                    }
                }
#pragma unroll
                for (int j = 0; j < RT; ++j) {
                    float2 &d = Cs[(q0r + j * (QT / RT)) * a.maxc + cc];
                    d.x += acc[j].x;
                    d.y += acc[j].y;
                }
            }
            __syncthreads();    // buffer c & 1 is refilled by the next pass
        }
        // 2. epilogue.  (a) screen every (q, nu) of the tile in FP32 (|x| <= 7 sigma plus a
        //    margin) and list the live ones, in item order, by a block-wide scan;
        //    (b) one live (q, nu) per thread: project on nu, rotate by U(k+q) for each
        //    surviving m (FP32 products), weights and occupations in FP64.  The list
        //    keeps whole warps on the projection however sparse the survivors are.
        double part = 0.0;
        const int64_t k = I.kidx[kb];
        const double en = I.eps[k * nw + n];
        const float en32 = I.eps32[k * nw + n];
        const double is = 1.0 / I.sigma, ycut2 = kDeltaCut * kDeltaCut;
        const float cut32 = (float)(kDeltaCut * I.sigma) + 1e-4f;
        for (int qq = t; qq < nq; qq += NT) kqrow[qq] = (int)kq_index(k, q0 + qq, I.kg, I.qg);
        __syncthreads();
        const int lane = t & 31, wid = t >> 5;
        int nlive = 0;
        for (int o0 = 0; o0 < QT * nm; o0 += NT) {
            const int o = o0 + t;
            uint32_t live = 0;
            if (o < QT * nm) {
                const int qq = o / nm, v = o - (o / nm) * nm;
                if (qq < nq) {
                    const int64_t q = q0 + qq;
                    const float w32 = I.hw32[q * nm + v];
                    if (w32 >= (float)kOmegaMinEv) {
                        const float *em32 = I.eps32 + (int64_t)kqrow[qq] * nw;
                        for (int m = 0; m < nw; ++m) {
                            const float d = en32 - em32[m];
                            if (fabsf(d - w32) <= cut32 || fabsf(d + w32) <= cut32) live |= 1u << m;
                        }
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, live != 0);
            if (lane == 0) wcnt[wid] = __popc(bal);
            __syncthreads();
            int base = nlive, tot = 0;
#pragma unroll
            for (int w2 = 0; w2 < NT / 32; ++w2) {
                base += (w2 < wid) ? wcnt[w2] : 0;
                tot += wcnt[w2];
            }
            if (live) items[base + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)o << 16) | live;
            nlive += tot;
            __syncthreads();
        }
        for (int j = t; j < nlive; j += NT) {
            const uint32_t it = items[j];
            uint32_t live = it & 0xffffu;
            const int o = (int)(it >> 16);
            const int qq = o / nm, v = o - (o / nm) * nm;
            const int64_t q = q0 + qq;
            const int64_t kq = kqrow[qq];
            const double w = I.hw[q * nm + v];
            const double *em = I.eps + kq * nw;
            const float2 *cf = I.coef + (q * nm + v) * nm;
            float2 gv[kMaxNw];
#pragma unroll
            for (int i = 0; i < kMaxNw; ++i) gv[i] = make_float2(0.f, 0.f);
            for (int ka = 0; ka < nm; ++ka) {
                const float2 cc = cf[ka];
                const float2 *row = Cs + qq * a.maxc + ka * nw;
#pragma unroll
                for (int i = 0; i < kMaxNw; ++i)
                    if (i < nw) cfma(gv[i], cc, row[i]);
            }
            const float2 *Ukq = I.U + kq * nw * nw;
            const double N = I.nbe[q * nm + v];
            while (live) {
                const int m = __ffs(live) - 1;
                live &= live - 1;
                float2 g = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < kMaxNw; ++i)
                    if (i < nw) cfma_conj(g, Ukq[m * nw + i], gv[i]);
                const double g2 = (double)cabs2(g);
                const double d = en - em[m];
                const double ye = (d - w) * is, ya = (d + w) * is;
                const double fm = I.focc[kq * nw + m];
                double W = 0.0;
                if (ye * ye <= ycut2) W += exp(-ye * ye) * (1.0 + N - fm);
                if (ya * ya <= ycut2) W += exp(-ya * ya) * (N + fm);
                part = fma(g2, W, part);
            }
        }
        // 3. block sum into this unit's slot (fixed tree)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
        if ((t & 31) == 0) red[t >> 5] = part;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w2 = 0; w2 < NT / 32; ++w2) s += red[w2];
            a.partial[u] = s;
        }
    }
}

// UT[k][m][i] = U[k][i][m]: the epilogue reads one final band m of U(k+q) per
// surviving term, so its nw values sit in two or four 32-byte sectors
__global__ void k_transpose_u(int64_t nk, int nw, const float2 *__restrict__ U, float2 *__restrict__ UT) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)nw * nw;
    if (t >= nk * per) return;
    const int64_t k = t / per;
    const int r = (int)(t % per), m = r / nw, i = r % nw;
    UT[t] = U[k * per + (int64_t)i * nw + m];
}

// Gamma rows: out[row] = scale * sum_qt partial[row * nqt + qt] for the rows of one instance
__global__ void k_batch_reduce(int nrows, int nqt, double scale, const double *__restrict__ partial,
                               double *__restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double s = 0.0;
    for (int i = 0; i < nqt; ++i) s += partial[(int64_t)r * nqt + i];
    out[r] = scale * s;
}

struct Cand {
    int qt, nt;
};
constexpr Cand kCands[4] = {{16, 128}, {32, 128}, {32, 256}, {64, 256}};

size_t smem_bytes(int qt, int maxc) { return sizeof(float2) * ((size_t)qt * maxc + 2 * ((size_t)qt * KC + (size_t)KC * maxc)); }

// CTAs per SM of a candidate (sets its shared-memory limit; call outside stream capture)
template <int QT, int NT>
cudaError_t prepare_one(int maxc, int *per_sm) {
    const size_t sh = smem_bytes(QT, maxc);
    cudaError_t e = cudaFuncSetAttribute(k_batch_rates<QT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_rates<QT, NT>, NT, sh);
    *per_sm = std::max(*per_sm, 1);
    return e;
}

cudaError_t prepare_cand(int ci, int maxc, int *per_sm) {
    switch (ci) {
        case 0: return prepare_one<16, 128>(maxc, per_sm);
        case 1: return prepare_one<32, 128>(maxc, per_sm);
        case 2: return prepare_one<32, 256>(maxc, per_sm);
        default: return prepare_one<64, 256>(maxc, per_sm);
    }
}

// persistent grid: every SM's resident CTAs, at most one per unit
cudaError_t launch_cand(int ci, const BArgs &a, cudaStream_t s, int nsm, int per_sm) {
    const int64_t grid = std::min<int64_t>((int64_t)nsm * per_sm, std::max<int64_t>(a.nunits, 1));
    const size_t sh = smem_bytes(kCands[ci].qt, a.maxc);
    switch (ci) {
        case 0: k_batch_rates<16, 128><<<(unsigned)grid, 128, sh, s>>>(a); break;
        case 1: k_batch_rates<32, 128><<<(unsigned)grid, 128, sh, s>>>(a); break;
        case 2: k_batch_rates<32, 256><<<(unsigned)grid, 256, sh, s>>>(a); break;
        default: k_batch_rates<64, 256><<<(unsigned)grid, 256, sh, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace

}  // namespace pgb

// ---------------------------------------------------------------------------
// host objects and the C ABI
// ---------------------------------------------------------------------------
using namespace pgb;

struct pgb_batch {
    std::vector<pgb_ctx *> ctx;
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 0;
    int maxc = 0;
    int cand = -1;                     // chosen candidate
    int prec = PGB_FP32;          // q-sum precision of the instances whose columns tile by 96
    int *d_err = nullptr;              // wait time-outs of the tensor-core q-sums
    float cand_ms[4] = {-1, -1, -1, -1};
    int per_sm[4] = {0, 0, 0, 0};      // resident CTAs per SM of each candidate
    int64_t graph_launches = 0;
    // arguments the graph was captured for
    std::vector<std::vector<int32_t>> kidx;
    std::vector<double> mu;
    double T = 0.0, sigma = 0.0;
    cudaGraphExec_t exec = nullptr;
    // device buffers owned by the batch
    std::vector<void *> bufs;
    BInst *d_inst = nullptr;
    int32_t *d_unit_inst = nullptr;
    double *d_partial = nullptr, *d_out = nullptr;
    int64_t nunits = 0, nout = 0;
    std::vector<int64_t> out0;         // first output row of each instance
    std::string err;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (void *p : bufs) cudaFree(p);
        bufs.clear();
        d_inst = nullptr;
        d_unit_inst = nullptr;
        d_partial = d_out = nullptr;
    }
};

namespace {

template <typename T>
pgb_status balloc(pgb_batch *b, T **p, size_t n) {
    void *x = nullptr;
    if (dev_malloc(&x, std::max<size_t>(n * sizeof(T), 16)) != cudaSuccess) {
        cudaGetLastError();
        b->err = "batch: device allocation failed";
        return PGB_ENOMEM;
    }
    b->bufs.push_back(x);
    *p = static_cast<T *>(x);
    return PGB_OK;
}

// Per-instance set-up plus the persistent kernel (and the reduction) on the
// batch stream; candidate ci.  Enqueue only: no allocation, no synchronisation.
struct Plan {
    std::vector<BInst> inst;
    struct Per {
        int32_t *kidx;
        void *phk, *S1, *G;
        double *focc, *nbe;
        float *eps32, *hw32;
        bool tc = false;               // q sum on the tensor cores (k_tc_qsum)
        int Kp = 0, ldc = 0;
        void *Asplit = nullptr, *Bsplit = nullptr;
        float2 *Ctc = nullptr;
    };
    std::vector<Per> per;
};

pgb_status enqueue(pgb_batch *b, Plan &P, int ci) {
    const int n = (int)b->ctx.size();
    if (b->prec != PGB_FP32 && cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream) != cudaSuccess) {
        b->err = "batch: error word reset failed";
        return PGB_ECUDA;
    }
    for (int i = 0; i < n; ++i) {
        pgb_ctx *c = b->ctx[i];
        cudaStream_t saved = c->stream;
        c->stream = b->stream;
        const int64_t nk = (int64_t)b->kidx[i].size();
        const int64_t ncol = (int64_t)c->nm * c->nw * c->nw;
        const int64_t nrowS = (int64_t)c->nRgp * ncol;
        Plan::Per &q = P.per[i];
        pgb_status st = launch_occ_tables(c, b->T, b->mu[i], q.focc, q.eps32, q.nbe, q.hw32);
        if (st == PGB_OK) st = launch_phase_grid(c, c->kg, q.kidx, nk, c->d_Rge, c->nRge, q.phk, true);
        if (st == PGB_OK)
            st = launch_cgemm(c, true, 1, nk, nrowS, c->nRge, q.phk, c->nRge, 0, c->d_g32, nrowS, 0, q.S1, nrowS, 0);
        if (st == PGB_OK) st = launch_fold_u(c, true, nk, q.kidx, c->nRgp, c->nm, c->nw, q.S1, c->d_U32, q.G);
        if (st == PGB_OK && q.tc) {
            const bool tf32 = b->prec == PGB_TC_TF32X3;
            st = launch_split_g(c, tf32, nk, c->nKp, (int)ncol, q.Kp, q.G, q.Bsplit, q.ldc);
            if (st == PGB_OK)
                st = launch_tc_qsum(c, tf32, nk, c->Nq, q.ldc, q.Kp, q.Asplit, q.Bsplit, q.Ctc, b->d_err);
        }
        c->stream = saved;
        if (st != PGB_OK) {
            b->err = "batch: set-up of instance " + std::to_string(i) + ": " + c->err;
            return st;
        }
    }
    BArgs a;
    a.ninst = n;
    a.inst = b->d_inst;
    a.unit_inst = b->d_unit_inst;
    a.nunits = b->nunits;
    a.maxc = b->maxc;
    a.partial = b->d_partial;
    cudaError_t e = launch_cand(ci, a, b->stream, b->nsm, b->per_sm[ci]);
    if (e != cudaSuccess) {
        b->err = std::string("batch: kernel launch: ") + cudaGetErrorString(e);
        return PGB_ECUDA;
    }
    for (int i = 0; i < n; ++i) {
        const BInst &I = P.inst[i];
        const int nrows = (int)(b->kidx[i].size() * I.nw);
        if (nrows == 0) continue;
        const double scale = kTwoPiOverHbar / ((double)I.Nq * b->sigma * kSqrtPi);
        k_batch_reduce<<<div_up(nrows, 128), 128, 0, b->stream>>>(nrows, I.nqt, scale, b->d_partial + I.unit0,
                                                                   b->d_out + b->out0[i]);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            b->err = std::string("batch: reduce launch: ") + cudaGetErrorString(e);
            return PGB_ECUDA;
        }
    }
    return PGB_OK;
}

pgb_status build_plan(pgb_batch *b, Plan &P, int qt) {
    const int n = (int)b->ctx.size();
    P.inst.assign(n, BInst());
    P.per.assign(n, Plan::Per());
    int64_t unit0 = 0, out0 = 0;
    b->out0.assign(n, 0);
    std::vector<int32_t> unit_inst;
    for (int i = 0; i < n; ++i) {
        pgb_ctx *c = b->ctx[i];
        const int64_t nk = (int64_t)b->kidx[i].size();
        const int64_t ncol = (int64_t)c->nm * c->nw * c->nw;
        BInst &I = P.inst[i];
        I.nw = c->nw;
        I.nm = c->nm;
        I.nRgp = c->nRgp;
        I.nKp = c->nKp;
        for (int d = 0; d < 3; ++d) {
            I.qg[d] = c->qg[d];
            I.kg[d] = c->kg[d];
        }
        I.Nq = c->Nq;
        I.nqt = (int)((c->Nq + qt - 1) / qt);
        I.unit0 = unit0;

        I.eps = c->d_eps;
        I.coef = c->d_coef32;
        I.hw = c->d_hw;
        I.sigma = b->sigma;
        Plan::Per &q = P.per[i];
        pgb_status st;
        if ((st = balloc(b, &q.kidx, (size_t)std::max<int64_t>(nk, 1))) != PGB_OK) return st;
        if (nk && cudaMemcpy(q.kidx, b->kidx[i].data(), 4 * (size_t)nk, cudaMemcpyHostToDevice) != cudaSuccess) {
            b->err = "batch: copy of k indices failed";
            return PGB_ECUDA;
        }
        char *phk, *S1, *G;
        if ((st = balloc(b, &phk, (size_t)nk * c->nRge * 8)) != PGB_OK) return st;
        if ((st = balloc(b, &S1, (size_t)nk * c->nRgp * ncol * 8)) != PGB_OK) return st;
        if ((st = balloc(b, &G, (size_t)nk * c->nKp * ncol * 8)) != PGB_OK) return st;
        q.phk = phk;
        q.S1 = S1;
        q.G = G;
        if ((st = balloc(b, &q.focc, (size_t)c->Nk * c->nw)) != PGB_OK) return st;
        if ((st = balloc(b, &q.eps32, (size_t)c->Nk * c->nw)) != PGB_OK) return st;
        if ((st = balloc(b, &q.nbe, (size_t)c->Nq * c->nm)) != PGB_OK) return st;
        if ((st = balloc(b, &q.hw32, (size_t)c->Nq * c->nm)) != PGB_OK) return st;
        // non-polar instances take the tensor-core q sum when the batch runs in a split
        // precision, their nm*nw*nw columns padded with zeros to a multiple of 96
        q.tc = b->prec != PGB_FP32 && !c->polar && nk > 0;
        float2 *phq = nullptr;
        if (q.tc) {
            const bool tf32 = b->prec == PGB_TC_TF32X3;
            const size_t tes = tf32 ? 4 : 2;
            q.Kp = tc_kpad(c->nKp);
            q.ldc = (int)((ncol + 95) / 96 * 96);
            char *As, *Bs;
            if ((st = balloc(b, &As, (size_t)4 * c->Nq * q.Kp * tes)) != PGB_OK) return st;
            if ((st = balloc(b, &Bs, (size_t)nk * 4 * q.ldc * q.Kp * tes)) != PGB_OK) return st;
            if ((st = balloc(b, &q.Ctc, (size_t)nk * c->Nq * q.ldc)) != PGB_OK) return st;
            q.Asplit = As;
            q.Bsplit = Bs;
            cudaStream_t saved = c->stream;   // split q phases: outside any capture
            c->stream = b->stream;
            st = launch_split_phases(c, tf32, c->qg, c->Nq, c->d_Rgp, c->nRgp, q.Kp, q.Asplit);
            c->stream = saved;
            if (st != PGB_OK || cudaStreamSynchronize(b->stream) != cudaSuccess) {
                b->err = "batch: split q phases of instance " + std::to_string(i) + " failed";
                return PGB_ECUDA;
            }
        } else {
            if ((st = balloc(b, &phq, (size_t)c->Nq * c->nKp)) != PGB_OK) return st;
            // q table, independent of the call's arguments: built here, outside any capture
            cudaStream_t saved = c->stream;
            c->stream = b->stream;
            st = launch_qtable_grid(c, nullptr, c->Nq, phq, true);
            c->stream = saved;
            if (st != PGB_OK || cudaStreamSynchronize(b->stream) != cudaSuccess) {
                b->err = "batch: q table of instance " + std::to_string(i) + " failed";
                return PGB_ECUDA;
            }
        }
        {   // transposed U table of the instance's k grid, outside any capture
            float2 *UT;
            if ((st = balloc(b, &UT, (size_t)c->Nk * c->nw * c->nw)) != PGB_OK) return st;
            const int64_t nt = c->Nk * c->nw * c->nw;
            k_transpose_u<<<div_up(nt, 256), 256, 0, b->stream>>>(c->Nk, c->nw, c->d_U32, UT);
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
                b->err = "batch: U transpose of instance " + std::to_string(i) + " failed";
                return PGB_ECUDA;
            }
            I.U = UT;
        }
        I.phq = phq;
        I.Ctc = q.Ctc;
        I.ldc = q.ldc;
        I.eps32 = q.eps32;
        I.hw32 = q.hw32;
        I.G = (const float2 *)G;
        I.kidx = q.kidx;
        I.focc = q.focc;
        I.nbe = q.nbe;
        const int64_t nu = nk * c->nw * I.nqt;
        unit_inst.insert(unit_inst.end(), (size_t)nu, i);
        unit0 += nu;
        b->out0[i] = out0;
        out0 += nk * c->nw;
    }
    b->nunits = unit0;
    b->nout = out0;
    pgb_status st;
    if ((st = balloc(b, &b->d_inst, (size_t)n)) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_unit_inst, (size_t)std::max<int64_t>(unit0, 1))) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_partial, (size_t)std::max<int64_t>(unit0, 1))) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_out, (size_t)std::max<int64_t>(out0, 1))) != PGB_OK) return st;
    if (cudaMemcpy(b->d_inst, P.inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        (unit0 && cudaMemcpy(b->d_unit_inst, unit_inst.data(), 4 * (size_t)unit0, cudaMemcpyHostToDevice) !=
                      cudaSuccess)) {
        b->err = "batch: descriptor upload failed";
        return PGB_ECUDA;
    }
    return PGB_OK;
}

}  // namespace

extern "C" {

pgb_status pgb_batch_create(pgb_batch **out, pgb_ctx *const *ctxs, int n) {
    if (!out || !ctxs || n <= 0) return PGB_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return PGB_EINVAL;
        if (!ctxs[i]->has_grids) {
            ctxs[i]->err = "batch_create: every context needs set_model and set_grids";
            return PGB_ESTATE;
        }
        if (ctxs[i]->device != ctxs[0]->device) {
            ctxs[i]->err = "batch_create: contexts must share one device";
            return PGB_EINVAL;
        }
    }
    pgb_batch *b = new pgb_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->device = ctxs[0]->device;
    cudaSetDevice(b->device);
    // a stream of its own: the legacy default stream cannot be captured
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return PGB_ECUDA;
    }
    if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        delete b;
        return PGB_ECUDA;
    }
    if (dev_malloc((void **)&b->d_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(b->stream);
        delete b;
        return PGB_ENOMEM;
    }
    for (int i = 0; i < n; ++i) b->maxc = std::max(b->maxc, ctxs[i]->nm * ctxs[i]->nw);
    for (int ci = 0; ci < 4; ++ci) {
        b->per_sm[ci] = 0;
        if (smem_bytes(kCands[ci].qt, b->maxc) > 220 * 1024) continue;   // does not fit: never tried
        if (prepare_cand(ci, b->maxc, &b->per_sm[ci]) != cudaSuccess) {
            cudaGetLastError();
            b->per_sm[ci] = 0;
        }
    }
    *out = b;
    return PGB_OK;
}

void pgb_batch_destroy(pgb_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->release();
    if (b->d_err) cudaFree(b->d_err);
    cudaStreamDestroy(b->stream);
    delete b;
}

pgb_status pgb_batch_set_precision(pgb_batch *b, int precision) {
    if (!b) return PGB_EINVAL;
    if (precision != PGB_FP32 && precision != PGB_TC_BF16X3 && precision != PGB_TC_TF32X3) {
        b->err = "batch_set_precision: PGB_FP32, PGB_TC_BF16X3 or PGB_TC_TF32X3";
        return PGB_EINVAL;
    }
    if (precision == b->prec) return PGB_OK;
    cudaSetDevice(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return PGB_ECUDA;
    if (precision != PGB_FP32) {   // function attributes are set here, outside any capture
        const pgb_status st = tc_qsum_prepare(b->ctx[0], precision == PGB_TC_TF32X3);
        if (st != PGB_OK) {
            b->err = "batch_set_precision: " + b->ctx[0]->err;
            return st;
        }
    }
    b->release();                        // the next call plans, tunes and captures again
    b->kidx.clear();
    b->prec = precision;
    b->cand = -1;
    for (float &m : b->cand_ms) m = -1.f;
    return PGB_OK;
}

const char *pgb_batch_last_error(const pgb_batch *b) { return b ? b->err.c_str() : "null batch"; }

pgb_status pgb_batch_rates(pgb_batch *b, const int32_t *const *k_idx, const int64_t *nk, double T_K,
                           const double *mu_eV, double sigma_eV, double *const *gamma_out) {
    if (!b) return PGB_EINVAL;
    cudaSetDevice(b->device);
    const int n = (int)b->ctx.size();
    if (!k_idx || !nk || !mu_eV || !gamma_out) {
        b->err = "batch_rates: null pointer";
        return PGB_EINVAL;
    }
    if (!(T_K > 0.0) || !(sigma_eV > 0.0)) {
        b->err = "batch_rates: need T > 0, sigma > 0";
        return PGB_EINVAL;
    }
    for (pgb_ctx *c : b->ctx)   // the members' own work (and host-side inputs) completes first
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            b->err = "batch_rates: a member stream failed";
            return PGB_ECUDA;
        }
    std::vector<std::vector<int32_t>> kk(n);
    std::vector<double> mu(mu_eV, mu_eV + n);
    for (int i = 0; i < n; ++i) {
        if (nk[i] < 0 || (nk[i] > 0 && (!k_idx[i] || !gamma_out[i]))) {
            b->err = "batch_rates: bad k list of instance " + std::to_string(i);
            return PGB_EINVAL;
        }
        if (!std::isfinite(mu[i])) {
            b->err = "batch_rates: non-finite mu";
            return PGB_EINVAL;
        }
        kk[i].resize(nk[i]);
        if (nk[i] && cudaMemcpy(kk[i].data(), k_idx[i], 4 * (size_t)nk[i], cudaMemcpyDefault) != cudaSuccess) {
            b->err = "batch_rates: k index copy failed";
            return PGB_ECUDA;
        }
        for (int32_t k : kk[i])
            if (k < 0 || k >= b->ctx[i]->Nk) {
                b->err = "batch_rates: k index out of range in instance " + std::to_string(i);
                return PGB_EINVAL;
            }
    }
    const bool same = b->exec && kk == b->kidx && mu == b->mu && T_K == b->T && sigma_eV == b->sigma;
    if (!same) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return PGB_ECUDA;
        b->release();
        b->kidx = kk;
        b->mu = mu;
        b->T = T_K;
        b->sigma = sigma_eV;
        // autotune on the first call: every candidate once, timed on the stream
        if (b->cand < 0) {
            float best = 1e30f;
            for (int ci = 0; ci < 4; ++ci) {
                if (b->per_sm[ci] <= 0) continue;
                Plan P;
                pgb_status st = build_plan(b, P, kCands[ci].qt);
                if (st != PGB_OK) return st;
                if ((st = enqueue(b, P, ci)) != PGB_OK) return st;   // warm-up
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, b->stream);
                st = enqueue(b, P, ci);
                cudaEventRecord(e1, b->stream);
                cudaError_t ce = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (st != PGB_OK) return st;
                if (ce != cudaSuccess) {
                    b->err = std::string("batch_rates: ") + cudaGetErrorString(ce);
                    return PGB_ECUDA;
                }
                b->cand_ms[ci] = ms;
                if (ms < best) {
                    best = ms;
                    b->cand = ci;
                }
                b->release();
            }
            if (b->cand < 0) {
                b->err = "batch_rates: no tile candidate fits in shared memory";
                return PGB_EINVAL;
            }
        }
        Plan P;
        pgb_status st = build_plan(b, P, kCands[b->cand].qt);
        if (st != PGB_OK) return st;
        // capture set-up, kernel and reduction in one graph
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            b->err = "batch_rates: stream capture could not start";
            return PGB_ECUDA;
        }
        st = enqueue(b, P, b->cand);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (st != PGB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess || cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->err = "batch_rates: graph capture failed";
            cudaGetLastError();
            return PGB_ECUDA;
        }
        cudaGraphDestroy(g);
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
        b->err = "batch_rates: graph launch failed";
        return PGB_ECUDA;
    }
    b->graph_launches++;
    for (int i = 0; i < n; ++i) {
        const size_t bytes = 8 * (size_t)kk[i].size() * b->ctx[i]->nw;
        if (bytes && cudaMemcpyAsync(gamma_out[i], b->d_out + b->out0[i], bytes, cudaMemcpyDefault, b->stream) !=
                         cudaSuccess) {
            b->err = "batch_rates: output copy failed";
            return PGB_ECUDA;
        }
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        b->err = "batch_rates: execution failed";
        return PGB_ECUDA;
    }
    if (b->prec != PGB_FP32) {
        int herr = 0;
        if (cudaMemcpy(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PGB_ECUDA;
        if (herr) {
            b->err = "batch_rates: a tensor-core pipeline wait ran out (bits " + std::to_string(herr) + ")";
            return PGB_ETIMEOUT;
        }
    }
    return PGB_OK;
}

pgb_status pgb_batch_tuning(const pgb_batch *b, int *tile_q, int *threads, float *cand_ms, int64_t *graph_launches) {
    if (!b) return PGB_EINVAL;
    if (tile_q) *tile_q = b->cand >= 0 ? kCands[b->cand].qt : 0;
    if (threads) *threads = b->cand >= 0 ? kCands[b->cand].nt : 0;
    if (cand_ms)
        for (int i = 0; i < 4; ++i) cand_ms[i] = b->cand_ms[i];
    if (graph_launches) *graph_launches = b->graph_launches;
    return PGB_OK;
}

}  // extern "C"
