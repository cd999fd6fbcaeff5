// Fused tensor-core scattering-rate kernel (Sec. 2.2.3 Eqs. eph_mat_wann2 and
// eph_mat; Sec. 2.1.2 Eqs. scatter_rate and BTE_W).
//
// For a batch of k-points it evaluates, per tile of 128 q x one pair of
// initial bands n:
//   mainloop (tensor cores): C[q][n][ka][i] = sum_p exp(i q.R_p) G_k[p][n][ka][i]
//     as four real products with hi/lo split operands (see tc_qsum.cu), FP32
//     accumulators in TMEM;
//   epilogue (CUDA cores, reading TMEM): per q row and band n, screen the
//     (m, nu) with |e_n(k) - e_m(k+q) -+ hw_nu(q)| <= 7 sigma, rotate by U(k+q)
//     once per surviving m (R_ka = sum_i conj(U_im) C[q][n][ka][i]), project on
//     the surviving modes (g = sum_ka coef[q][nu][ka] R_ka), and accumulate
//     |g|^2 [e^{-(x_em/s)^2}(1 + N - f_m) + e^{-(x_abs/s)^2}(N + f_m)].
// The per-tile sums over q go to partial[b][q-tile][nu][n]; a second kernel
// reduces the q-tiles in a fixed order.
//
// Persistent CTAs (one per SM) walk the tiles in k-groups so that a group's
// operands stay in L2.  Warp roles: 0 = TMA producer, 1 = TMEM owner and MMA
// issuer, 2-9 = epilogue (warp w reads TMEM lane group w % 4, one q row per
// thread, for one of the tile's two bands).  With BF16x3
// the two accumulators (re, im) are double-buffered in TMEM so the epilogue of
// one tile overlaps the mainloop of the next; TF32x3 keeps separate
// correction accumulators (four per tile, single-buffered).
#include <algorithm>
#include <cstdio>

#include <cudaTypedefs.h>

#include "internal.cuh"
#include "tc.cuh"
#include "weights.cuh"

namespace pgb {

namespace {

constexpr int BM = 128;
constexpr int BN = 96;                    // complex columns per tile
constexpr int STAGES = 3;
constexpr int ROWB = 64;
constexpr int A_PART = BM * ROWB;
constexpr int B_PART = BN * ROWB;
// B stage regions (hi, lo): rows [-Bi | Br | Bi], so [Br; Bi] (rows 96..287) and
// [-Bi; Br] (rows 0..191) are both contiguous 192-row MMA operands
constexpr int B_REGION = 3 * B_PART;
constexpr int STAGE_BYTES = 4 * A_PART + 2 * B_REGION;
constexpr int MN = 2 * BN;                // MMA N: re and im columns together
constexpr long long WAIT_BUDGET = 1ll << 31;
constexpr int NWF = 8, NMF = 6;           // band and mode counts of this kernel
constexpr int PER_N = NWF * NMF;          // 48 columns per initial band
constexpr int NPT = BN / PER_N;           // 2 bands per tile
constexpr int NPAIR = NWF / NPT;          // 4 tiles per (k, q-tile)

template <bool TF32> struct Cfg;
template <> struct Cfg<false> { static constexpr int NACC = 2, BUFS = 2; };
template <> struct Cfg<true> { static constexpr int NACC = 4, BUFS = 1; };

constexpr int NEPI = 8;                          // epilogue warps: 4 lane groups x 2 bands
constexpr int NTHREADS = 64 + 32 * NEPI;
constexpr int NBARS = 2 * STAGES + 2 * 2 + 1;   // full, empty, acc_full[2], acc_empty[2], drain
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;

struct FusedArgs {
    int nb, Nq, Nk, Kp, nqt, gk;
    const int32_t *kidx;
    int kg[3], qg[3];
    // per-grid-point tables, grid index fastest so that a warp's 32
    // consecutive q (and nearly consecutive k+q) read whole sectors
    const float2 *ehl;     // [NW][Nk] shifted band energy as (hi, lo) floats
    const float *focc;     // [NW][Nk]
    const float2 *UT;      // [m][i][Nk]
    const float2 *coef;    // [nu][ka][Nq]
    const float2 *whl;     // [NM][Nq] hbar*omega as (hi, lo) floats
    const float *nbe;      // [NM][Nq]
    float inv_sigma;
    float cut;             // screening bound on |x|, eV
    double *partial;       // [nb][nqt][NM][NW]
    int *err;
};

// Work unit = (k, q-tile); a CTA runs the NPAIR band-pair tiles of a unit back
// to back.  Units are ordered in k-groups of gk so a group's operands stay in L2.
__device__ __forceinline__ void decode_unit(int unit, int nb, int nqt, int gk, int &b, int &qt) {
    const int per_group = gk * nqt;
    const int g = unit / per_group;
    const int rem = unit - g * per_group;
    const int gsize = min(gk, nb - g * gk);
    const int kk = rem % gsize;
    qt = rem / gsize;
    b = g * gk + kk;
}

template <bool TF32>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_rates(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, FusedArgs a) {
    constexpr int NACC = Cfg<TF32>::NACC, BUFS = Cfg<TF32>::BUFS;
    constexpr int TMEM_COLS = 512;
    static_assert(NACC * BN * BUFS <= TMEM_COLS, "TMEM budget");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *full = bars, *empty = bars + STAGES, *accf = bars + 2 * STAGES, *acce = accf + 2,
             *drain = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *red = reinterpret_cast<float *>(tmem_slot + 4);    // [NEPI warps][NM]
    volatile int *stopv = reinterpret_cast<volatile int *>(red + NEPI * NMF);   // [NEPI]

    __shared__ int skip;
    if (threadIdx.x == 0) skip = *reinterpret_cast<volatile int *>(a.err);
    __syncthreads();
    if (skip) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int EK = TF32 ? 16 : 32;
    constexpr int KSTEP = TF32 ? 8 : 16;
    const int nk = a.Kp / EK;
    const int nunits = a.nb * a.nqt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(tc::smem_addr(full + s), 1);
            tc::mbar_init(tc::smem_addr(empty + s), 1);
        }
        for (int u = 0; u < 2; ++u) {
            tc::mbar_init(tc::smem_addr(accf + u), 1);
            tc::mbar_init(tc::smem_addr(acce + u), NEPI);
        }
        tc::mbar_init(tc::smem_addr(drain), 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        tc::prefetch_tmap(&tA);
        tc::prefetch_tmap(&tB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_addr(tmem_slot), TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------ TMA producer ------------------------------
        int it = 0;
        for (int tile = blockIdx.x * NPAIR; tile < nunits * NPAIR && !*abort_flag;
             tile += (tile % NPAIR == NPAIR - 1) ? (gridDim.x - 1) * NPAIR + 1 : 1) {
            int b, qt;
            decode_unit(tile / NPAIR, a.nb, a.nqt, a.gk, b, qt);
            const int np = tile % NPAIR;
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % STAGES;
                if (it >= STAGES &&
                    !tc::mbar_wait(tc::smem_addr(empty + s), ((it / STAGES) - 1) & 1, WAIT_BUDGET)) {
                    atomicOr(a.err, 1);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                const uint32_t fb = tc::smem_addr(full + s);
                tc::mbar_expect_tx(fb, STAGE_BYTES);
                uint8_t *st = smem + s * STAGE_BYTES;
                for (int p = 0; p < 4; ++p)
                    tc::tma_load_3d(tc::smem_addr(st + p * A_PART), &tA, fb, kc * EK, qt * BM, p);
                // B parts in global memory: 0 Br_hi, 1 Br_lo, 2 Bi_hi, 3 Bi_lo, 4 -Bi_hi, 5 -Bi_lo
                uint8_t *bh = st + 4 * A_PART, *bl = bh + B_REGION;
                uint8_t *dstp[6] = {bh + B_PART, bl + B_PART, bh + 2 * B_PART, bl + 2 * B_PART, bh, bl};
                for (int p = 0; p < 6; ++p)
                    tc::tma_load_3d(tc::smem_addr(dstp[p]), &tB, fb, kc * EK, np * BN, b * 6 + p);
            }
        }
        for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
            tc::mbar_wait(tc::smem_addr(full + j % STAGES), (j / STAGES) & 1, WAIT_BUDGET);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------ MMA issuer ------------------------------
        constexpr uint32_t fmt = TF32 ? 2u : 1u;
        constexpr uint32_t idp = tc::make_idesc(fmt, BM, MN, false);
        int it = 0, tl = 0;
        for (int tile = blockIdx.x * NPAIR; tile < nunits * NPAIR && !*abort_flag;
             tile += (tile % NPAIR == NPAIR - 1) ? (gridDim.x - 1) * NPAIR + 1 : 1, ++tl) {
            const int buf = tl % BUFS;
            if (tl >= BUFS && !tc::mbar_wait(tc::smem_addr(acce + buf), ((tl / BUFS) - 1) & 1, 4 * WAIT_BUDGET)) {
                atomicOr(a.err, 2);
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t d0 = tbase + buf * NACC * BN;
            // [re | im] main accumulator; TF32 keeps the corrections in a second one
            const uint32_t d_main = d0, d_corr = (NACC == 4) ? d0 + MN : d0;
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % STAGES;
                if (!tc::mbar_wait(tc::smem_addr(full + s), (it / STAGES) & 1, WAIT_BUDGET) || *abort_flag) {
                    atomicOr(a.err, 2);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t st = tc::smem_addr(smem + s * STAGE_BYTES);
#pragma unroll
                for (int ks = 0; ks < EK / KSTEP; ++ks) {
                    const uint32_t off = ks * 32;
                    const uint64_t arh = tc::desc_sw64(st + 0 * A_PART + off);
                    const uint64_t arl = tc::desc_sw64(st + 1 * A_PART + off);
                    const uint64_t aih = tc::desc_sw64(st + 2 * A_PART + off);
                    const uint64_t ail = tc::desc_sw64(st + 3 * A_PART + off);
                    const uint32_t bh = st + 4 * A_PART + off, bl = bh + B_REGION;
                    const uint64_t b1h = tc::desc_sw64(bh + B_PART), b1l = tc::desc_sw64(bl + B_PART);   // [Br; Bi]
                    const uint64_t b2h = tc::desc_sw64(bh), b2l = tc::desc_sw64(bl);                     // [-Bi; Br]
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    const uint32_t acc_c = (NACC == 4) ? acc : 1u;
                    // [C_re | C_im] += Ar [Br | Bi] + Ai [-Bi | Br]
                    tc::mma<TF32>(d_main, arh, b1h, idp, acc);
                    tc::mma<TF32>(d_main, aih, b2h, idp, 1);
                    tc::mma<TF32>(d_corr, arh, b1l, idp, acc_c);
                    tc::mma<TF32>(d_corr, arl, b1h, idp, 1);
                    tc::mma<TF32>(d_corr, aih, b2l, idp, 1);
                    tc::mma<TF32>(d_corr, ail, b2h, idp, 1);
                }
                tc::mma_commit(tc::smem_addr(empty + s));
            }
            if (!ok) break;
            tc::mma_commit(tc::smem_addr(accf + buf));
        }
        tc::mma_commit(tc::smem_addr(drain));
        tc::mbar_wait(tc::smem_addr(drain), 0, WAIT_BUDGET);
    } else if (warp >= 2) {
        // ------------------------------ epilogue ------------------------------
        // thread = (q row of the tile, band n = 2 np + nl); all arithmetic FP32:
        // x = ((e_n,hi - e_m,hi) - w_hi) + ((e_n,lo - e_m,lo) - w_lo), where the
        // shifted energies make e_n,hi - e_m,hi exact for every term that can
        // survive the screen.
        const int ew = warp - 2;
        const int lg = warp & 3;
        const int nl = ew / 4;
        const int row = lg * 32 + lane;
        const uint32_t lane_off = (uint32_t)(lg * 32) << 16;
        const int kg2 = a.kg[2], kg1 = a.kg[1], kg0 = a.kg[0];
        const int qg2 = a.qg[2], qg1 = a.qg[1];
        const int s0 = kg0 / a.qg[0], s1 = kg1 / qg1, s2 = kg2 / qg2;
        int tl = 0;
        int cur_unit = -1;
        int k = 0, q = 0, kq = 0;
        bool valid = false;
        float2 em[NWF], wv[NMF];
        float nb_[NMF];
        for (int tile = blockIdx.x * NPAIR; tile < nunits * NPAIR;
             tile += (tile % NPAIR == NPAIR - 1) ? (gridDim.x - 1) * NPAIR + 1 : 1, ++tl) {
            const int unit = tile / NPAIR, np = tile % NPAIR;
            int b, qt;
            decode_unit(unit, a.nb, a.nqt, a.gk, b, qt);
            if (unit != cur_unit) {
                // per-(k, q) data, kept in registers for the unit's four tiles;
                // loaded before the accumulator wait so the latency overlaps the MMAs
                cur_unit = unit;
                k = a.kidx[b];
                q = qt * BM + row;
                valid = q < a.Nq;
                if (valid) {
                    const int k3 = k % kg2, k2 = (k / kg2) % kg1, k1 = k / (kg1 * kg2);
                    const int q3 = q % qg2, q2 = (q / qg2) % qg1, q1 = q / (qg1 * qg2);
                    int t1 = k1 + q1 * s0, t2 = k2 + q2 * s1, t3 = k3 + q3 * s2;
                    t1 -= (t1 >= kg0) ? kg0 : 0;
                    t2 -= (t2 >= kg1) ? kg1 : 0;
                    t3 -= (t3 >= kg2) ? kg2 : 0;
                    kq = (t1 * kg1 + t2) * kg2 + t3;
#pragma unroll
                    for (int m = 0; m < NWF; ++m) em[m] = a.ehl[(size_t)m * a.Nk + kq];
#pragma unroll
                    for (int v = 0; v < NMF; ++v) {
                        wv[v] = a.whl[(size_t)v * a.Nq + q];
                        nb_[v] = a.nbe[(size_t)v * a.Nq + q];
                    }
                }
            }
            const int buf = tl % BUFS;
            bool ok = tc::mbar_wait(tc::smem_addr(accf + buf), (tl / BUFS) & 1, 8 * WAIT_BUDGET);
            ok = __all_sync(0xffffffffu, ok);
            // one stop decision for all epilogue warps, from values written before the barrier
            if (lane == 0) stopv[ew] = (!ok || *abort_flag) ? 1 : 0;
            if (!ok && lane == 0) {
                atomicOr(a.err, 4);
                *abort_flag = 1;
            }
            tc::named_sync(1, 32 * NEPI);
            int stop = 0;
#pragma unroll
            for (int w8 = 0; w8 < NEPI; ++w8) stop |= stopv[w8];
            if (stop) break;
            tc::fence_after_sync();
            const int n = np * NPT + nl;
            const uint32_t tb = tbase + lane_off + buf * NACC * BN + nl * PER_N;
            float gr[PER_N], gi[PER_N];
            tc::tmem_ld48(tb, gr);
            tc::tmem_ld48(tb + BN, gi);
            if constexpr (NACC == 4) {
                float cr[PER_N];
                tc::tmem_ld48(tb + 2 * BN, cr);
#pragma unroll
                for (int j = 0; j < PER_N; ++j) gr[j] += cr[j];
                tc::tmem_ld48(tb + 3 * BN, cr);
#pragma unroll
                for (int j = 0; j < PER_N; ++j) gi[j] += cr[j];
            }
            // the accumulator buffer can be refilled as soon as it has been read
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_addr(acce + buf));

            float acc[NMF];
#pragma unroll
            for (int v = 0; v < NMF; ++v) acc[v] = 0.f;
            if (valid) {
                const float2 en = a.ehl[(size_t)n * a.Nk + k];
                // screen every (nu, m) first; live[nu] holds the surviving m
                uint32_t live[NMF], any = 0;
#pragma unroll
                for (int v = 0; v < NMF; ++v) {
                    live[v] = 0;
                    if (!(wv[v].x + wv[v].y >= (float)kOmegaMinEv)) continue;
#pragma unroll
                    for (int m = 0; m < NWF; ++m) {
                        // (e_n,hi - e_m,hi) is exact for every possible survivor
                        const float dh = en.x - em[m].x, dl = en.y - em[m].y;
                        const float xe = mismatch32(dh, dl, wv[v], -1.f);
                        const float xa = mismatch32(dh, dl, wv[v], 1.f);
                        if (fabsf(xe) <= a.cut || fabsf(xa) <= a.cut) live[v] |= 1u << m;
                    }
                    any |= live[v];
                }
                // g_mn^nu = sum_ka coef[nu][ka] R_ka with R_ka = sum_i conj(U_im(k+q)) C[ka][i]:
                // the rotation runs once per surviving m, the projection once per surviving (m, nu)
                while (any) {
                    const int m = __ffs(any) - 1;
                    any &= any - 1;
                    float2 u[NWF];
#pragma unroll
                    for (int i = 0; i < NWF; ++i) u[i] = a.UT[(size_t)(m * NWF + i) * a.Nk + kq];
                    const float f = a.focc[(size_t)m * a.Nk + kq];
                    float rr[NMF], ri[NMF];
#pragma unroll
                    for (int ka = 0; ka < NMF; ++ka) {
                        float sr = 0.f, si = 0.f;
#pragma unroll
                        for (int i = 0; i < NWF; ++i) {
                            const float xr = gr[ka * NWF + i], xi = gi[ka * NWF + i];
                            sr = fmaf(u[i].x, xr, fmaf(u[i].y, xi, sr));
                            si = fmaf(u[i].x, xi, fmaf(-u[i].y, xr, si));
                        }
                        rr[ka] = sr;
                        ri[ka] = si;
                    }
                    const float dh = en.x - em[m].x, dl = en.y - em[m].y;
#pragma unroll
                    for (int v = 0; v < NMF; ++v) {
                        if (!((live[v] >> m) & 1u)) continue;
                        float grr = 0.f, gii = 0.f;
#pragma unroll
                        for (int ka = 0; ka < NMF; ++ka) {
                            const float2 c = a.coef[(size_t)(v * NMF + ka) * a.Nq + q];
                            grr = fmaf(c.x, rr[ka], fmaf(-c.y, ri[ka], grr));
                            gii = fmaf(c.x, ri[ka], fmaf(c.y, rr[ka], gii));
                        }
                        const float g2 = grr * grr + gii * gii;
                        const float xe = mismatch32(dh, dl, wv[v], -1.f);
                        const float xa = mismatch32(dh, dl, wv[v], 1.f);
                        const float N = nb_[v];
                        float W = 0.f;
                        if (fabsf(xe) <= a.cut) W += gauss32(xe, a.inv_sigma) * (1.f + N - f);
                        if (fabsf(xa) <= a.cut) W += gauss32(xa, a.inv_sigma) * (N + f);
                        acc[v] = fmaf(g2, W, acc[v]);
                    }
                }
            }
            // sum over the tile's 128 q rows: warp shuffle, then the four warps of this band
#pragma unroll
            for (int v = 0; v < NMF; ++v) {
                float x = acc[v];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) red[ew * NMF + v] = x;
            }
            tc::named_sync(1, 32 * NEPI);
            if ((ew & 3) == 0 && lane < NMF) {
                const int v = lane;
                double sum = 0.0;
                for (int w4 = 0; w4 < 4; ++w4) sum += (double)red[(nl * 4 + w4) * NMF + v];
                a.partial[(((size_t)b * a.nqt + qt) * NMF + v) * NWF + n] = sum;
            }
            tc::named_sync(1, 32 * NEPI);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, TMEM_COLS);
    }
}

int make_map3(CUtensorMap *m, void *base, bool tf32, int Kp, int64_t d1, int64_t d2, int box_rows) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return -1;
        }
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    const int esz = tf32 ? 4 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)d1, (cuuint64_t)d2};
    const cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)Kp * esz * d1};
    const cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return (int)enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace

bool tc_fused_supported(int nw, int nm) { return nw == NWF && nm == NMF; }

namespace {
// The fused epilogue's arithmetic for single terms: shift and split the FP64
// energies as the tables do, then the mismatch, the screen and the weight.
__global__ void k_diag_delta(int64_t n, const double *__restrict__ en, const double *__restrict__ em,
                             const double *__restrict__ hw, double eps_ref, float inv_sigma, float cut,
                             float *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float2 a = split_hl(en[t] - eps_ref), b = split_hl(em[t] - eps_ref), w = split_hl(hw[t]);
    const float dh = a.x - b.x, dl = a.y - b.y;
    const float xe = mismatch32(dh, dl, w, -1.f), xa = mismatch32(dh, dl, w, 1.f);
    out[4 * t + 0] = xe;
    out[4 * t + 1] = xa;
    out[4 * t + 2] = fabsf(xe) <= cut ? gauss32(xe, inv_sigma) : 0.f;
    out[4 * t + 3] = fabsf(xa) <= cut ? gauss32(xa, inv_sigma) : 0.f;
}
}  // namespace

pgb_status diag_delta_weights(pgb_ctx *c, int64_t n, const double *en, const double *em, const double *hw,
                              double eps_ref, double sigma, float *out) {
    if (n == 0) return PGB_OK;
    k_diag_delta<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, en, em, hw, eps_ref, (float)(1.0 / sigma),
                                                                     (float)(kDeltaCut * sigma), out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_tc_rates(pgb_ctx *c, bool tf32, const FusedLaunch &L) {
    if (L.nb == 0) return PGB_OK;
    const int nqt = (int)((c->Nq + BM - 1) / BM);
    CUtensorMap tA, tB;
    const int ra = make_map3(&tA, c->d_asplit, tf32, L.Kp, c->Nq, 4, BM);
    const int rb = ra == 0 ? make_map3(&tB, L.Bsplit, tf32, L.Kp, NWF * NMF * NWF, L.nb * 6, BN) : 0;
    if (ra != 0 || rb != 0) {
        c->err = "fused tensor-core rates: cuTensorMapEncodeTiled failed (A " + std::to_string(ra) + ", B " +
                 std::to_string(rb) + ")";
        return PGB_ECUDA;
    }
    FusedArgs a;
    a.nb = (int)L.nb;
    a.Nq = (int)c->Nq;
    a.Nk = (int)c->Nk;
    a.Kp = L.Kp;
    a.nqt = nqt;
    a.gk = std::max(1, std::min<int>(16, (int)L.nb));
    a.kidx = L.kidx;
    for (int d = 0; d < 3; ++d) {
        a.kg[d] = c->kg[d];
        a.qg[d] = c->qg[d];
    }
    a.ehl = L.ehl;
    a.focc = L.focc32;
    a.UT = c->d_U32T;
    a.coef = c->d_coefT;
    a.whl = L.whl;
    a.nbe = L.nbe32;
    a.inv_sigma = (float)(1.0 / L.sigma);
    a.cut = (float)(kDeltaCut * L.sigma);
    a.partial = L.partial;
    a.err = c->d_err;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t nunits = L.nb * (int64_t)nqt;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nunits, sms > 0 ? sms : 148));
    if (tf32) {
        PGB_CUDA_TRY(c, cudaFuncSetAttribute(k_tc_rates<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        k_tc_rates<true><<<grid, NTHREADS, SMEM_BYTES, c->stream>>>(tA, tB, a);
    } else {
        PGB_CUDA_TRY(c, cudaFuncSetAttribute(k_tc_rates<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        k_tc_rates<false><<<grid, NTHREADS, SMEM_BYTES, c->stream>>>(tA, tB, a);
    }
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb
