// Scattering rates (Eqs. scatter_rate, BTE_W) of many independent model
// instances of uneven band, mode and grid sizes in one persistent launch.
//
// Each member context holds its own model and grids.  Per call, the per-
// instance set-up and one persistent kernel over the work units of every
// instance are captured in a CUDA graph, which later calls with the same
// arguments replay.
//
// Per instance (set-up, in the graph): occupation tables, the R_e sums with
// U(k) folded for its k list, and the R_p sums
//   C[b][q][n ka i] = sum_p e^{iq.R_p} G_kb[p][n ka i]
// over its whole q grid (FP32 form: the SIMT complex GEMM; BF16x3 / TF32x3:
// tcgen05 on split operands, columns padded to a multiple of 96), written to
// HBM once.
//
// Persistent kernel, one warp per task: a chunk of qc q-points of one (instance,
// k), every band n of the instance in turn.  For each (q, n) row the warp reads
// the row of C into registers (coalesced; nm*nw complex values, up to eight per
// lane), screens the (nu, m) of the row 32 at a time against |x| <= 7 sigma
// (FP32 with a margin), and evaluates each live term as a warp-wide dot product
//   g_mn nu = sum_{ka, i} coef[q][nu][ka] conj(U_im(k+q)) C[q][n][ka][i]
// (FP32 products, shuffle reduction).  Live terms wait in lane slots, 32 at a
// time, so that their energy differences, Gaussian weights and occupation
// factors are taken in FP64 by full warps; each band's sum over the chunk goes
// to its own partial slot.  Warps claim chunks from a counter in order of
// decreasing cost (instances with the most work per chunk first), so the uneven
// instances balance over the SMs; a second kernel adds the chunk partials of
// each (instance, k, n) in order, so results do not depend on the schedule.
//
// The chunk length and the block size are chosen by a small autotuner: on the
// first call every candidate runs once, timed with events, and the fastest is
// kept.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "cplx.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

struct BInst {
    int nw, nm;
    int qg[3], kg[3];
    int64_t Nq;
    int qc;                    // q-points per chunk
    int nch;                   // chunks per k
    int ib;                    // lanes per mode column in a row's dot product (nm * ib <= 32, ib divides nw)
    int64_t chunk0;            // first chunk of this instance in the claim order
    int64_t part0;             // first partial: [nk][nw][nch]
    const float2 *C;           // [nk][Nq][ldc] R_p sums with U(k) folded, columns (n, ka, i)
    int64_t ldc;
    const int32_t *kidx;       // [nk]
    const double *eps;         // [Nk][nw]
    const float *eps32;        // [Nk][nw] FP32 copy for the screen
    const float2 *U;           // [Nk][m][i] transposed: row m of U(k) contiguous
    const float2 *coef;        // [Nq][nu][ka]
    const double *hw;          // [Nq][nm]
    const float *hw32;         // [Nq][nm] FP32 copy for the screen
    const double *focc;        // [Nk][nw]
    const double *nbe;         // [Nq][nm]
    double sigma;
};

struct BArgs {
    const BInst *inst;
    const int32_t *chunk_inst; // [nchunks] instance of each chunk, costliest instances first
    int64_t nchunks;
    unsigned long long *next;  // chunk counter, zeroed before each launch
    double *partial;
};

constexpr int kTPL = (kMaxNw * kMaxNmode + 31) / 32;   // row elements per lane (8)

// One chunk of one instance: q-points q0 .. q0 + nq of k-point b, every band.
// sum_i conj(U_im) C[ka][i] over this lane's EL elements
template <int EL>
__device__ __forceinline__ float2 rot_part(const float2 *__restrict__ ur, const float2 (&cr)[kMaxNw]) {
    float2 rr = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < EL; ++e) cfma_conj(rr, ur[e], cr[e]);
    return rr;
}

__device__ __forceinline__ float2 rot_dispatch(int el, const float2 *__restrict__ ur, const float2 (&cr)[kMaxNw]) {
    switch (el) {
        case 1: return rot_part<1>(ur, cr);
        case 2: return rot_part<2>(ur, cr);
        case 3: return rot_part<3>(ur, cr);
        case 4: return rot_part<4>(ur, cr);
        case 6: return rot_part<6>(ur, cr);
        case 8: return rot_part<8>(ur, cr);
        case 12: return rot_part<12>(ur, cr);
        default: {
            float2 rr = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < kMaxNw; ++e)
                if (e < el) cfma_conj(rr, ur[e], cr[e]);
            return rr;
        }
    }
}

__device__ __forceinline__ void batch_chunk(const BInst &I, int64_t b, int qci, double *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int nw = I.nw, nm = I.nm, P = nm * nw, nc = nm * nw;
    const int64_t q0 = (int64_t)qci * I.qc;
    const int nq = (int)(I.Nq - q0 < I.qc ? I.Nq - q0 : I.qc);
    const int64_t k = I.kidx[b];
    // grid coordinates of k and of the chunk's first q; k+q follows q incrementally
    const int kg0 = I.kg[0], kg1 = I.kg[1], kg2 = I.kg[2], qg1 = I.qg[1], qg2 = I.qg[2];
    const int st0 = kg0 / I.qg[0], st1 = kg1 / qg1, st2 = kg2 / qg2;
    const int k3 = (int)(k % kg2), k2 = (int)((k / kg2) % kg1), k1 = (int)(k / ((int64_t)kg1 * kg2));
    int c3 = (int)(q0 % qg2), c2 = (int)((q0 / qg2) % qg1), c1 = (int)(q0 / ((int64_t)qg1 * qg2));
    // lane -> (mode column ka, block of EL consecutive i) of a row: ib lanes per ka
    const int ib = I.ib, el = nw / ib;
    const bool act = lane < nm * ib;
    const int ka = act ? lane / ib : 0, i0 = act ? (lane - (lane / ib) * ib) * el : 0;
    // screen combos c = 32 j + lane -> (m, nu), m-major so that the live terms of one final
    // band m arrive together and share its rotation; packed as nu * 16 + m, four per word
    uint32_t scm[kTPL / 4] = {0u, 0u};
#pragma unroll
    for (int j = 0; j < kTPL; ++j) {
        const int cc = 32 * j + lane;
        const uint32_t m = cc < nc ? (uint32_t)(cc / nm) : 0u, v = cc < nc ? (uint32_t)(cc - (cc / nm) * nm) : 0u;
        scm[j / 4] |= ((v << 4) | m) << (8 * (j % 4));
    }
    const int nj = (nc + 31) / 32;
    const double is = 1.0 / I.sigma, ycut2 = kDeltaCut * kDeltaCut;
    const float cut32 = (float)(kDeltaCut * I.sigma) + 1e-4f;
    // band energies at k: band n in lane n
    const float en32_l = lane < nw ? I.eps32[k * nw + lane] : 0.f;
    const double en64_l = lane < nw ? I.eps[k * nw + lane] : 0.0;
    double acc = 0.0;   // lane n: band n's sum over the chunk
    // the term waiting in this lane's slot: |g|^2, band n, and the indices of e_m(k+q) and (q, nu)
    int pending = 0, p_n = 0, p_e = 0, p_qv = 0;
    float p_g2 = 0.f;
    // weights of the waiting terms in FP64 (full warp), then per-band sums in a fixed order
    auto flush = [&](int count) {
        double contrib = 0.0;
        const double en = __shfl_sync(0xffffffffu, en64_l, p_n);
        if (lane < count) {
            const double w = I.hw[p_qv], N = I.nbe[p_qv], f = I.focc[p_e];
            const double d = en - I.eps[p_e];
            const double ye = (d - w) * is, ya = (d + w) * is;
            double W = 0.0;
            if (ye * ye <= ycut2) W += exp(-ye * ye) * (1.0 + N - f);
            if (ya * ya <= ycut2) W += exp(-ya * ya) * (N + f);
            contrib = (double)p_g2 * W;
        }
        // per-band sums of the (at most 32) waiting terms in FP32, only over the bands present;
        // the chunk's band sums accumulate in FP64
        double mine = 0.0;
        unsigned todo = 0u;
        for (int nn = 0; nn < nw; ++nn) todo |= __ballot_sync(0xffffffffu, lane < count && p_n == nn) ? (1u << nn) : 0u;
        while (todo) {
            const int nn = __ffs(todo) - 1;
            todo &= todo - 1;
            float sh = (lane < count && p_n == nn) ? (float)contrib : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sh += __shfl_xor_sync(0xffffffffu, sh, o);
            if (lane == nn) mine = (double)sh;
        }
        acc += mine;
    };
    for (int qq = 0; qq < nq; ++qq) {
        const int64_t q = q0 + qq;
        int t1 = k1 + c1 * st0, t2 = k2 + c2 * st1, t3 = k3 + c3 * st2;
        t1 -= (t1 >= kg0) ? kg0 : 0;
        t2 -= (t2 >= kg1) ? kg1 : 0;
        t3 -= (t3 >= kg2) ? kg2 : 0;
        const int kq = (t1 * kg1 + t2) * kg2 + t3;
        if (++c3 == qg2) {
            c3 = 0;
            if (++c2 == qg1) {
                c2 = 0;
                ++c1;
            }
        }
        // screening inputs held by lanes: e_m(k+q) in lane m, hbar*omega_nu(q) in lane nu
        const float em_l = lane < nw ? I.eps32[(int64_t)kq * nw + lane] : 0.f;
        const float w_l = lane < nm ? I.hw32[q * nm + lane] : 0.f;
        const float2 *Ukq = I.U + (int64_t)kq * nw * nw + i0;
        const float2 *cq = I.coef + q * nm * nm + ka;
        for (int n = 0; n < nw; ++n) {
            const float en = __shfl_sync(0xffffffffu, en32_l, n);
            bool loaded = false;
            int m_rot = -1;   // final band whose rotation rr_m holds (this row)
            float2 rr_m = make_float2(0.f, 0.f);
            float2 cr[kMaxNw];
            for (int j = 0; j < nj; ++j) {
                const uint32_t vm = (scm[j / 4] >> (8 * (j % 4))) & 0xffu;
                const float em = __shfl_sync(0xffffffffu, em_l, (int)(vm & 15u));
                const float w = __shfl_sync(0xffffffffu, w_l, (int)(vm >> 4));
                bool live = false;
                if (32 * j + lane < nc && w >= (float)kOmegaMinEv) {
                    const float d = en - em;
                    live = fabsf(d - w) <= cut32 || fabsf(d + w) <= cut32;
                }
                unsigned bal = __ballot_sync(0xffffffffu, live);
                if (bal && !loaded) {
                    // this lane's elements C[q][n][ka][i0 .. i0 + EL), loaded once the row has a live term
                    const float2 *crow = I.C + (b * I.Nq + q) * I.ldc + (int64_t)n * P + ka * nw + i0;
#pragma unroll
                    for (int e = 0; e < kMaxNw; ++e) cr[e] = (act && e < el) ? crow[e] : make_float2(0.f, 0.f);
                    loaded = true;
                }
                while (bal) {
                    // up to four live terms at a time, so their loads and reductions overlap
                    constexpr int TB = 4;
                    int cnt = 0;
                    uint32_t tv[TB];
#pragma unroll
                    for (int u = 0; u < TB; ++u) {
                        const int src = bal ? __ffs(bal) - 1 : 0;
                        tv[u] = __shfl_sync(0xffffffffu, vm, src);
                        if (bal) {
                            bal &= bal - 1;
                            ++cnt;
                        }
                    }
                    // g = sum_ka coef[q][nu][ka] sum_i conj(U_im(k+q)) C[q][n][ka][i]
                    float2 g[TB];
#pragma unroll
                    for (int u = 0; u < TB; ++u) {
                        g[u] = make_float2(0.f, 0.f);
                        if (u < cnt) {   // warp-uniform
                            const int v = (int)(tv[u] >> 4), m = (int)(tv[u] & 15u);
                            if (m != m_rot) {   // the rotation of final band m, once per run of its terms
                                rr_m = act ? rot_dispatch(el, Ukq + m * nw, cr) : make_float2(0.f, 0.f);
                                m_rot = m;
                            }
                            if (act) cfma(g[u], cq[v * nm], rr_m);
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                        for (int u = 0; u < TB; ++u) {
                            g[u].x += __shfl_xor_sync(0xffffffffu, g[u].x, o);
                            g[u].y += __shfl_xor_sync(0xffffffffu, g[u].y, o);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < TB; ++u) {
                        if (u >= cnt) break;
                        if (lane == pending) {
                            p_n = n;
                            p_g2 = cabs2(g[u]);
                            p_e = kq * nw + (int)(tv[u] & 15u);
                            p_qv = (int)(q * nm) + (int)(tv[u] >> 4);
                        }
                        if (++pending == 32) {
                            flush(32);
                            pending = 0;
                        }
                    }
                }
            }
        }
    }
    flush(pending);
    if (lane < nw) partial[I.part0 + (b * nw + lane) * I.nch + qci] = acc;
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_batch_warp(BArgs a) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(a.next, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((long long)c >= a.nchunks) break;
        const BInst &I = a.inst[a.chunk_inst[c]];
        const int64_t r = (int64_t)c - I.chunk0;
        const int qci = (int)(r % I.nch);
        const int64_t b = r / I.nch;
        batch_chunk(I, b, qci, a.partial);
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

// Autotuner candidates: block size and a scale of the chunk length.
struct Cand {
    int nt;
    int scale;
};
constexpr Cand kCands[4] = {{256, 1}, {256, 4}, {512, 4}, {512, 16}};

// q-points per chunk: about 4096 lane-steps of work per band at scale 1.
int pick_qc(int scale, int nw, int nm) {
    const int want = 4096 / (nw * (nm * nw + 32));
    int qc = 8;
    while (qc * 2 <= want && qc < 512) qc *= 2;
    return qc * scale;
}

template <int NT>
cudaError_t prepare_one(int *per_sm) {
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_warp<NT>, NT, 0);
    *per_sm = std::max(*per_sm, 1);
    return e;
}

// CTAs per SM of a candidate (call outside stream capture)
cudaError_t prepare_cand(int ci, int *per_sm) {
    switch (kCands[ci].nt) {
        case 128: return prepare_one<128>(per_sm);
        case 256: return prepare_one<256>(per_sm);
        default: return prepare_one<512>(per_sm);
    }
}

// persistent grid: every SM's resident CTAs, at most one warp per chunk
cudaError_t launch_cand(int ci, const BArgs &a, cudaStream_t s, int nsm, int per_sm) {
    const int nt = kCands[ci].nt;
    const int64_t grid = std::min<int64_t>((int64_t)nsm * per_sm, std::max<int64_t>((a.nchunks + nt / 32 - 1) / (nt / 32), 1));
    switch (nt) {
        case 128: k_batch_warp<128><<<(unsigned)grid, 128, 0, s>>>(a); break;
        case 256: k_batch_warp<256><<<(unsigned)grid, 256, 0, s>>>(a); break;
        default: k_batch_warp<512><<<(unsigned)grid, 512, 0, s>>>(a); break;
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
    int cand = -1;                     // chosen candidate
    int prec = PGB_FP32;               // q-sum precision: SIMT FP32 or tensor-core split
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
    int32_t *d_chunk_inst = nullptr;
    double *d_partial = nullptr, *d_out = nullptr;
    unsigned long long *d_next = nullptr;
    int64_t nchunks = 0, nout = 0;
    std::vector<int64_t> out0;         // first output row of each instance
    std::vector<int> qc;               // chunk length of each instance for the current candidate
    std::string err;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (void *p : bufs) cudaFree(p);
        bufs.clear();
        d_inst = nullptr;
        d_chunk_inst = nullptr;
        d_partial = d_out = nullptr;
        d_next = nullptr;
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

// Per-instance buffers and tables of one call (independent of the tile candidate).
struct Plan {
    std::vector<BInst> inst;
    struct Per {
        int32_t *kidx = nullptr;
        void *phk = nullptr, *S1 = nullptr, *G = nullptr;
        double *focc = nullptr, *nbe = nullptr;
        float *eps32 = nullptr, *hw32 = nullptr;
        float2 *phq = nullptr;         // FP32 q table (SIMT q-sum)
        bool tc = false;               // q-sum on the tensor cores (k_tc_qsum)
        int Kp = 0;
        int64_t ldc = 0;
        void *Asplit = nullptr, *Bsplit = nullptr;
        float2 *C = nullptr;           // [nk][Nq][ldc]
    };
    std::vector<Per> per;
};

// Enqueue the set-up of every instance, the persistent kernel of candidate ci and
// the reductions on the batch stream.  No allocation, no synchronisation.
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
        if (nk > 0) {
            if (st == PGB_OK) st = launch_phase_grid(c, c->kg, q.kidx, nk, c->d_Rge, c->nRge, q.phk, true);
            if (st == PGB_OK)
                st = launch_cgemm(c, true, 1, nk, nrowS, c->nRge, q.phk, c->nRge, 0, c->d_g32, nrowS, 0, q.S1, nrowS, 0);
            if (st == PGB_OK) st = launch_fold_u(c, true, nk, q.kidx, c->nRgp, c->nm, c->nw, q.S1, c->d_U32, q.G);
            if (st == PGB_OK && q.tc) {
                const bool tf32 = b->prec == PGB_TC_TF32X3;
                st = launch_split_g(c, tf32, nk, c->nKp, (int)ncol, q.Kp, q.G, q.Bsplit, (int)q.ldc);
                if (st == PGB_OK)
                    st = launch_tc_qsum(c, tf32, nk, c->Nq, (int)q.ldc, q.Kp, q.Asplit, q.Bsplit, q.C, b->d_err);
            } else if (st == PGB_OK) {
                st = launch_cgemm(c, true, nk, c->Nq, ncol, c->nKp, q.phq, c->nKp, 0, q.G, ncol, (int64_t)c->nKp * ncol,
                                  q.C, ncol, c->Nq * ncol);
            }
        }
        c->stream = saved;
        if (st != PGB_OK) {
            b->err = "batch: set-up of instance " + std::to_string(i) + ": " + c->err;
            return st;
        }
    }
    if (cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), b->stream) != cudaSuccess) {
        b->err = "batch: chunk counter reset failed";
        return PGB_ECUDA;
    }
    BArgs a;
    a.inst = b->d_inst;
    a.chunk_inst = b->d_chunk_inst;
    a.nchunks = b->nchunks;
    a.next = b->d_next;
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
        k_batch_reduce<<<div_up(nrows, 128), 128, 0, b->stream>>>(nrows, I.nch, scale, b->d_partial + I.part0,
                                                                   b->d_out + b->out0[i]);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            b->err = std::string("batch: reduce launch: ") + cudaGetErrorString(e);
            return PGB_ECUDA;
        }
    }
    return PGB_OK;
}

// Buffers and call-independent tables of every instance (q tables or split q phases,
// transposed U), built outside any capture.
pgb_status build_plan(pgb_batch *b, Plan &P) {
    const int n = (int)b->ctx.size();
    P.inst.assign(n, BInst());
    P.per.assign(n, Plan::Per());
    int64_t out0 = 0;
    b->out0.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        pgb_ctx *c = b->ctx[i];
        const int64_t nk = (int64_t)b->kidx[i].size();
        const int64_t ncol = (int64_t)c->nm * c->nw * c->nw;
        BInst &I = P.inst[i];
        I.nw = c->nw;
        I.nm = c->nm;
        for (int d = 0; d < 3; ++d) {
            I.qg[d] = c->qg[d];
            I.kg[d] = c->kg[d];
        }
        I.Nq = c->Nq;
        I.ib = 1;
        for (int ib : {4, 2})
            if (I.ib == 1 && c->nm * ib <= 32 && c->nw % ib == 0) I.ib = ib;
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
        // split precisions: every instance's q-sum on the tensor cores, its nm*nw*nw
        // columns padded with zeros to a multiple of 96 (polar instances carry the
        // long-range term in nm extra rows of the split phases)
        q.tc = b->prec != PGB_FP32 && nk > 0;
        cudaStream_t saved = c->stream;
        c->stream = b->stream;
        if (q.tc) {
            const bool tf32 = b->prec == PGB_TC_TF32X3;
            const size_t tes = tf32 ? 4 : 2;
            q.Kp = tc_kpad(c->nKp);
            q.ldc = (ncol + 95) / 96 * 96;
            char *As, *Bs;
            if ((st = balloc(b, &As, (size_t)4 * c->Nq * q.Kp * tes)) == PGB_OK &&
                (st = balloc(b, &Bs, (size_t)nk * 4 * q.ldc * q.Kp * tes)) == PGB_OK) {
                q.Asplit = As;
                q.Bsplit = Bs;
                st = launch_split_phases(c, tf32, c->qg, c->Nq, c->d_Rgp, c->nRgp, q.Kp, q.Asplit, c->d_polarL,
                                         c->polar ? c->nm : 0);
            }
        } else {
            q.ldc = ncol;
            if ((st = balloc(b, &q.phq, (size_t)c->Nq * c->nKp)) == PGB_OK)
                st = launch_qtable_grid(c, nullptr, c->Nq, q.phq, true);
        }
        c->stream = saved;
        if (st == PGB_OK) st = balloc(b, &q.C, (size_t)std::max<int64_t>(nk, 1) * c->Nq * q.ldc);
        if (st != PGB_OK || cudaStreamSynchronize(b->stream) != cudaSuccess) {
            if (b->err.empty() || st == PGB_OK) b->err = "batch: q tables of instance " + std::to_string(i) + " failed";
            return st != PGB_OK ? st : PGB_ECUDA;
        }
        {   // transposed U table of the instance's k grid
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
        I.C = q.C;
        I.ldc = q.ldc;
        I.eps32 = q.eps32;
        I.hw32 = q.hw32;
        I.kidx = q.kidx;
        I.focc = q.focc;
        I.nbe = q.nbe;
        b->out0[i] = out0;
        out0 += nk * c->nw;
    }
    b->nout = out0;
    pgb_status st;
    if ((st = balloc(b, &b->d_out, (size_t)std::max<int64_t>(out0, 1))) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_next, 1)) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_inst, (size_t)n)) != PGB_OK) return st;
    return PGB_OK;
}

// Chunk lengths, chunk order and partial slots of candidate ci; uploads the descriptors.
pgb_status set_candidate(pgb_batch *b, Plan &P, int ci) {
    const int n = (int)b->ctx.size();
    b->qc.assign(n, 0);
    std::vector<double> cost(n, 0.0);
    int64_t part0 = 0;
    for (int i = 0; i < n; ++i) {
        BInst &I = P.inst[i];
        I.qc = pick_qc(kCands[ci].scale, I.nw, I.nm);
        b->qc[i] = I.qc;
        I.nch = (int)((I.Nq + I.qc - 1) / I.qc);
        I.part0 = part0;
        part0 += (int64_t)b->kidx[i].size() * I.nw * I.nch;
        cost[i] = (double)I.qc * I.nw * (I.nm * I.nw + 32);
    }
    // chunks of the costliest instances first, so the counter hands out the big ones early
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<int32_t> chunk_inst;
    int64_t chunk0 = 0;
    for (int i : order) {
        BInst &I = P.inst[i];
        I.chunk0 = chunk0;
        const int64_t nch = (int64_t)b->kidx[i].size() * I.nch;
        chunk_inst.insert(chunk_inst.end(), (size_t)nch, i);
        chunk0 += nch;
    }
    b->nchunks = chunk0;
    pgb_status st;
    if ((st = balloc(b, &b->d_chunk_inst, (size_t)std::max<int64_t>(chunk0, 1))) != PGB_OK) return st;
    if ((st = balloc(b, &b->d_partial, (size_t)std::max<int64_t>(part0, 1))) != PGB_OK) return st;
    if (cudaMemcpy(b->d_inst, P.inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        (chunk0 && cudaMemcpy(b->d_chunk_inst, chunk_inst.data(), 4 * (size_t)chunk0, cudaMemcpyHostToDevice) !=
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
        cudaStreamDestroy(b->stream);
        delete b;
        return PGB_ECUDA;
    }
    if (dev_malloc((void **)&b->d_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(b->stream);
        delete b;
        return PGB_ENOMEM;
    }
    for (int ci = 0; ci < 4; ++ci) {
        if (prepare_cand(ci, &b->per_sm[ci]) != cudaSuccess) {
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
        Plan P;
        pgb_status st = build_plan(b, P);
        if (st != PGB_OK) {
            b->release();
            b->kidx.clear();
            return st;
        }
        // autotune on the first call: every candidate once (after a warm-up), timed on the stream
        if (b->cand < 0) {
            float best = 1e30f;
            for (int ci = 0; ci < 4; ++ci) {
                if (b->per_sm[ci] <= 0) continue;
                if ((st = set_candidate(b, P, ci)) != PGB_OK) break;
                if ((st = enqueue(b, P, ci)) != PGB_OK) break;   // warm-up
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
                if (st != PGB_OK) break;
                if (ce != cudaSuccess) {
                    b->err = std::string("batch_rates: ") + cudaGetErrorString(ce);
                    st = PGB_ECUDA;
                    break;
                }
                b->cand_ms[ci] = ms;
                if (ms < best) {
                    best = ms;
                    b->cand = ci;
                }
            }
            if (st == PGB_OK && b->cand < 0) {
                b->err = "batch_rates: no candidate could be launched";
                st = PGB_EINVAL;
            }
            if (st != PGB_OK) {
                b->release();
                b->kidx.clear();
                b->cand = -1;
                return st;
            }
        }
        if ((st = set_candidate(b, P, b->cand)) != PGB_OK) {
            b->release();
            b->kidx.clear();
            return st;
        }
        // capture set-up, kernel and reduction in one graph
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            b->err = "batch_rates: stream capture could not start";
            b->release();
            b->kidx.clear();
            return PGB_ECUDA;
        }
        st = enqueue(b, P, b->cand);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (st != PGB_OK || ce != cudaSuccess || cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (st == PGB_OK) b->err = "batch_rates: graph capture failed";
            cudaGetLastError();
            b->release();
            b->kidx.clear();
            return st != PGB_OK ? st : PGB_ECUDA;
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
    if (tile_q) *tile_q = b->qc.empty() ? 0 : *std::max_element(b->qc.begin(), b->qc.end());
    if (threads) *threads = b->cand >= 0 ? kCands[b->cand].nt : 0;
    if (cand_ms)
        for (int i = 0; i < 4; ++i) cand_ms[i] = b->cand_ms[i];
    if (graph_launches) *graph_launches = b->graph_launches;
    return PGB_OK;
}

}  // extern "C"
