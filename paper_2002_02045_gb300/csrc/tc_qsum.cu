// Tensor-core q-sum of the e-ph interpolation (Sec. 2.2.3, Eq. eph_mat_wann2):
//   C[b][q][c] = sum_p exp(i q.R_p) G[b][p][c]            (complex, per k = b)
// on tcgen05 with TMA-staged operands and FP32 accumulators in TMEM.
//
// The complex product is four real products, C_re = Ar Br - Ai Bi and
// C_im = Ar Bi + Ai Br, and each real operand x is split into x_hi + x_lo
// (BF16 or TF32); x*y is formed as hi*hi + hi*lo + lo*hi (three MMAs).  The
// minus sign of Ai Bi is the instruction descriptor's negate-A bit.  The
// tensor core's FP32 accumulation is biased toward zero by a fraction of an
// ulp per accumulate step, so the large hi*hi products and the small
// hi*lo + lo*hi corrections go to separate accumulators (four 96-column
// TMEM accumulators: re, im, re correction, im correction) that the epilogue
// adds in FP32 with round-to-nearest; the large ones then see a third of the
// accumulate steps.
//
// Operand layouts (K = R_p padded to Kp, K-major, 64-byte swizzled tiles):
//   A: [4][Nq][Kp] parts (Ar_hi, Ar_lo, Ai_hi, Ai_lo), shared by every k;
//   B: [nb][4][ncol][Kp] parts (Br_hi, Br_lo, Bi_hi, Bi_lo) per k.
// One CTA computes a 128 (q) x 96 (c) complex tile of one k: warp 0 issues
// TMA loads into a 3-stage ring, warp 1 owns TMEM and issues the MMAs, warps
// 2-5 read the two 96-column accumulators (re, im) and store C.
#include <climits>
#include <cstdio>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "internal.cuh"
#include "tc.cuh"

namespace pgb {

namespace {

constexpr int BM = 128;              // q rows per tile
constexpr int BN = 96;               // complex columns per tile
constexpr int STAGES = 3;
constexpr int ROWB = 64;             // bytes per swizzled row (64-byte swizzle)
constexpr int A_PART = BM * ROWB;    // 8192
constexpr int B_PART = BN * ROWB;    // 6144
constexpr int STAGE_BYTES = 4 * A_PART + 4 * B_PART;   // 57344
constexpr int TMEM_COLS = 512;       // re, im, re correction, im correction at 0, 96, 192, 288
constexpr long long WAIT_BUDGET = 1ll << 31;           // ~1 s of clock cycles
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct TcArgs {
    int64_t Nq;       // rows of C (q-points of this launch)
    int q_off;        // first row of the A table that this launch multiplies
    int Kp;
    int ncol;
    int nb;
    float2 *C;        // [nb][Nq][ncol]
    int *err;         // error bits: 1 producer, 2 mma, 4 epilogue wait ran out
};

template <bool TF32>
__global__ void __launch_bounds__(192, 1)
    k_tc_qsum(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    // bars[0..S) full, bars[S..2S) empty, bars[2S] accumulator ready, bars[2S+1] drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    // another CTA already hit a time-out: the whole CTA leaves before touching TMEM
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *reinterpret_cast<volatile int *>(a.err);
    __syncthreads();
    if (skip) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN;
    const int q0 = blockIdx.y * BM;
    const int b = blockIdx.z;
    constexpr int EK = TF32 ? 16 : 32;          // K elements per 64-byte row
    constexpr int KSTEP = TF32 ? 8 : 16;        // K per MMA (32 bytes)
    const int nk = a.Kp / EK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * STAGES + 2; ++s) tc::mbar_init(tc::smem_addr(bars + s), 1);
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
        // ---------------- TMA producer ----------------
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            if (kc >= STAGES && !tc::mbar_wait(tc::smem_addr(bars + STAGES + s), ((kc / STAGES) - 1) & 1, WAIT_BUDGET)) {
                atomicOr(a.err, 1);
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const uint32_t full = tc::smem_addr(bars + s);
            tc::mbar_expect_tx(full, STAGE_BYTES);
            uint8_t *st = smem + s * STAGE_BYTES;
            for (int p = 0; p < 4; ++p)
                tc::tma_load_3d(tc::smem_addr(st + p * A_PART), &tA, full, kc * EK, a.q_off + q0, p);
            for (int p = 0; p < 4; ++p)
                tc::tma_load_3d(tc::smem_addr(st + 4 * A_PART + p * B_PART), &tB, full, kc * EK, n0, b * 4 + p);
            ++issued;
        }
        // let the loads still in flight land before the CTA can exit
        for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
            tc::mbar_wait(tc::smem_addr(bars + kc % STAGES), (kc / STAGES) & 1, WAIT_BUDGET);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t fmt = TF32 ? 2u : 1u;
        constexpr uint32_t idp = tc::make_idesc(fmt, BM, BN, false);
        constexpr uint32_t idn = tc::make_idesc(fmt, BM, BN, true);
        const uint32_t d_re = tbase, d_im = tbase + BN, d_rec = tbase + 2 * BN, d_imc = tbase + 3 * BN;
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            if (!tc::mbar_wait(tc::smem_addr(bars + s), (kc / STAGES) & 1, WAIT_BUDGET) || *abort_flag) {
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
                const uint64_t arh = tc::desc_sw64(st + 0 * A_PART + off), arl = tc::desc_sw64(st + 1 * A_PART + off);
                const uint64_t aih = tc::desc_sw64(st + 2 * A_PART + off), ail = tc::desc_sw64(st + 3 * A_PART + off);
                const uint32_t bb = st + 4 * A_PART + off;
                const uint64_t brh = tc::desc_sw64(bb + 0 * B_PART), brl = tc::desc_sw64(bb + 1 * B_PART);
                const uint64_t bih = tc::desc_sw64(bb + 2 * B_PART), bil = tc::desc_sw64(bb + 3 * B_PART);
                const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                // C_re += Ar Br - Ai Bi   (hi*hi terms | hi*lo + lo*hi terms)
                tc::mma<TF32>(d_re, arh, brh, idp, acc);
                tc::mma<TF32>(d_re, aih, bih, idn, 1);
                tc::mma<TF32>(d_rec, arh, brl, idp, acc);
                tc::mma<TF32>(d_rec, arl, brh, idp, 1);
                tc::mma<TF32>(d_rec, aih, bil, idn, 1);
                tc::mma<TF32>(d_rec, ail, bih, idn, 1);
                // C_im += Ar Bi + Ai Br
                tc::mma<TF32>(d_im, arh, bih, idp, acc);
                tc::mma<TF32>(d_im, aih, brh, idp, 1);
                tc::mma<TF32>(d_imc, arh, bil, idp, acc);
                tc::mma<TF32>(d_imc, arl, bih, idp, 1);
                tc::mma<TF32>(d_imc, aih, brl, idp, 1);
                tc::mma<TF32>(d_imc, ail, brh, idp, 1);
            }
            tc::mma_commit(tc::smem_addr(bars + STAGES + s));   // frees the stage when these MMAs finish
        }
        if (ok) tc::mma_commit(tc::smem_addr(bars + 2 * STAGES));
        // drain: every MMA of this thread has finished before TMEM is released
        tc::mma_commit(tc::smem_addr(bars + 2 * STAGES + 1));
        tc::mbar_wait(tc::smem_addr(bars + 2 * STAGES + 1), 0, WAIT_BUDGET);
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> registers -> C ----------------
        const bool ready = tc::mbar_wait(tc::smem_addr(bars + 2 * STAGES), 0, 4 * WAIT_BUDGET);
        if (!ready) atomicOr(a.err, 4);
        tc::fence_after_sync();
        const int lg = warp & 3;                  // TMEM lane group of this warp
        const int row = lg * 32 + lane;
        const int64_t q = (int64_t)q0 + row;
        const uint32_t lane_addr = tbase + ((uint32_t)(lg * 32) << 16);
        float2 *crow = a.C + ((int64_t)b * a.Nq + q) * a.ncol + n0;
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ++ch) {
            float re[32], im[32], cr[32];
            tc::tmem_ld32(lane_addr + ch * 32, re);
            tc::tmem_ld32(lane_addr + 2 * BN + ch * 32, cr);
#pragma unroll
            for (int j = 0; j < 32; ++j) re[j] += cr[j];
            tc::tmem_ld32(lane_addr + BN + ch * 32, im);
            tc::tmem_ld32(lane_addr + 3 * BN + ch * 32, cr);
#pragma unroll
            for (int j = 0; j < 32; ++j) im[j] += cr[j];
            if (ready && q < a.Nq) {
                float4 *dst = reinterpret_cast<float4 *>(crow + ch * 32);
#pragma unroll
                for (int j = 0; j < 16; ++j) dst[j] = make_float4(re[2 * j], im[2 * j], re[2 * j + 1], im[2 * j + 1]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, TMEM_COLS);
    }
}

// TF32x3 form with chunked accumulation.  The tensor core adds each MMA's
// products to its FP32 accumulator with truncation, ~0.6 ulp of the
// accumulator toward zero per instruction on these sums, so a single
// accumulator over the whole K (96 instructions per real part at K = 384)
// shrinks |C| by a few 1e-6 (|g|^2 by ~1.4e-5).  Here every chunk of 32 K
// elements (4 MMA K-steps) starts a fresh accumulator, double-buffered in TMEM
// (re, im: 2 x 96 columns per buffer), and the epilogue warps add the chunk
// values into FP32 registers with round-to-nearest while the next chunk is
// multiplied.  Each accumulator then sees 24 instructions on a partial sum of
// 32 terms, and the chunk errors add with random signs: about 4x less error.
constexpr int TF_CHUNK_STAGES = 2;          // stages (16 K elements each) per chunk
constexpr int TF_NEPI = 8;                  // epilogue warps: 4 lane groups x 2 column halves
constexpr int TF_THREADS = 64 + 32 * TF_NEPI;

__global__ void __launch_bounds__(TF_THREADS, 1)
    k_tc_qsum_tf32(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    // full[S], empty[S], accf[2] (chunk ready), acce[2] (chunk drained), drain
    uint64_t *full = bars, *empty = bars + STAGES, *accf = bars + 2 * STAGES, *acce = accf + 2, *drain = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    __shared__ int skip;
    if (threadIdx.x == 0) skip = *reinterpret_cast<volatile int *>(a.err);
    __syncthreads();
    if (skip) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN;
    const int q0 = blockIdx.y * BM;
    const int b = blockIdx.z;
    constexpr int EK = 16, KSTEP = 8;
    const int nk = a.Kp / EK;
    const int nchunk = (nk + TF_CHUNK_STAGES - 1) / TF_CHUNK_STAGES;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            tc::mbar_init(tc::smem_addr(full + st), 1);
            tc::mbar_init(tc::smem_addr(empty + st), 1);
        }
        for (int u = 0; u < 2; ++u) {
            tc::mbar_init(tc::smem_addr(accf + u), 1);
            tc::mbar_init(tc::smem_addr(acce + u), TF_NEPI);
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
        // ---------------- TMA producer ----------------
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int st = kc % STAGES;
            if (kc >= STAGES && !tc::mbar_wait(tc::smem_addr(empty + st), ((kc / STAGES) - 1) & 1, WAIT_BUDGET)) {
                atomicOr(a.err, 1);
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const uint32_t fb = tc::smem_addr(full + st);
            tc::mbar_expect_tx(fb, STAGE_BYTES);
            uint8_t *sp = smem + st * STAGE_BYTES;
            for (int p = 0; p < 4; ++p) tc::tma_load_3d(tc::smem_addr(sp + p * A_PART), &tA, fb, kc * EK, a.q_off + q0, p);
            for (int p = 0; p < 4; ++p)
                tc::tma_load_3d(tc::smem_addr(sp + 4 * A_PART + p * B_PART), &tB, fb, kc * EK, n0, b * 4 + p);
            ++issued;
        }
        for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
            tc::mbar_wait(tc::smem_addr(full + kc % STAGES), (kc / STAGES) & 1, WAIT_BUDGET);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idp = tc::make_idesc(2u, BM, BN, false);
        constexpr uint32_t idn = tc::make_idesc(2u, BM, BN, true);
        bool ok = true;
        for (int ch = 0; ch < nchunk && ok; ++ch) {
            const int buf = ch & 1;
            if (ch >= 2 && !tc::mbar_wait(tc::smem_addr(acce + buf), ((ch >> 1) - 1) & 1, 4 * WAIT_BUDGET)) {
                atomicOr(a.err, 2);
                *abort_flag = 1;
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t d_re = tbase + buf * 2 * BN, d_im = d_re + BN;
            const int kc1 = min(nk, (ch + 1) * TF_CHUNK_STAGES);
            for (int kc = ch * TF_CHUNK_STAGES; kc < kc1; ++kc) {
                const int st = kc % STAGES;
                if (!tc::mbar_wait(tc::smem_addr(full + st), (kc / STAGES) & 1, WAIT_BUDGET) || *abort_flag) {
                    atomicOr(a.err, 2);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t sp = tc::smem_addr(smem + st * STAGE_BYTES);
#pragma unroll
                for (int ks = 0; ks < EK / KSTEP; ++ks) {
                    const uint32_t off = ks * 32;
                    const uint64_t arh = tc::desc_sw64(sp + 0 * A_PART + off), arl = tc::desc_sw64(sp + 1 * A_PART + off);
                    const uint64_t aih = tc::desc_sw64(sp + 2 * A_PART + off), ail = tc::desc_sw64(sp + 3 * A_PART + off);
                    const uint32_t bb = sp + 4 * A_PART + off;
                    const uint64_t brh = tc::desc_sw64(bb + 0 * B_PART), brl = tc::desc_sw64(bb + 1 * B_PART);
                    const uint64_t bih = tc::desc_sw64(bb + 2 * B_PART), bil = tc::desc_sw64(bb + 3 * B_PART);
                    const uint32_t acc = (kc > ch * TF_CHUNK_STAGES || ks > 0) ? 1u : 0u;
                    // C_re += Ar Br - Ai Bi, C_im += Ar Bi + Ai Br (hi*hi, hi*lo, lo*hi)
                    tc::mma<true>(d_re, arh, brh, idp, acc);
                    tc::mma<true>(d_re, aih, bih, idn, 1);
                    tc::mma<true>(d_re, arh, brl, idp, 1);
                    tc::mma<true>(d_re, arl, brh, idp, 1);
                    tc::mma<true>(d_re, aih, bil, idn, 1);
                    tc::mma<true>(d_re, ail, bih, idn, 1);
                    tc::mma<true>(d_im, arh, bih, idp, acc);
                    tc::mma<true>(d_im, aih, brh, idp, 1);
                    tc::mma<true>(d_im, arh, bil, idp, 1);
                    tc::mma<true>(d_im, arl, bih, idp, 1);
                    tc::mma<true>(d_im, aih, brl, idp, 1);
                    tc::mma<true>(d_im, ail, brh, idp, 1);
                }
                tc::mma_commit(tc::smem_addr(empty + st));
            }
            if (ok) tc::mma_commit(tc::smem_addr(accf + buf));
        }
        tc::mma_commit(tc::smem_addr(drain));
        tc::mbar_wait(tc::smem_addr(drain), 0, WAIT_BUDGET);
    } else if (warp >= 2) {
        // ---------------- epilogue: per chunk TMEM -> FP32 register sums ----------------
        const int ew = warp - 2;
        const int lg = warp & 3;               // TMEM lane group of this warp
        const int half = ew >> 2;              // columns [48 half, 48 half + 48)
        const int row = lg * 32 + lane;
        const int64_t q = (int64_t)q0 + row;
        const uint32_t lane_addr = tbase + ((uint32_t)(lg * 32) << 16) + half * (BN / 2);
        float sr[BN / 2], si[BN / 2];
#pragma unroll
        for (int j = 0; j < BN / 2; ++j) sr[j] = si[j] = 0.f;
        bool ok = true;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int buf = ch & 1;
            ok = tc::mbar_wait(tc::smem_addr(accf + buf), (ch >> 1) & 1, 4 * WAIT_BUDGET);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicOr(a.err, 4);
                break;
            }
            tc::fence_after_sync();
            float v[BN / 2];
            tc::tmem_ld48(lane_addr + buf * 2 * BN, v);
#pragma unroll
            for (int j = 0; j < BN / 2; ++j) sr[j] += v[j];
            tc::tmem_ld48(lane_addr + buf * 2 * BN + BN, v);
#pragma unroll
            for (int j = 0; j < BN / 2; ++j) si[j] += v[j];
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_addr(acce + buf));
        }
        if (ok && q < a.Nq) {
            float4 *dst = reinterpret_cast<float4 *>(a.C + ((int64_t)b * a.Nq + q) * a.ncol + n0 + half * (BN / 2));
#pragma unroll
            for (int j = 0; j < BN / 4; ++j) dst[j] = make_float4(sr[2 * j], si[2 * j], sr[2 * j + 1], si[2 * j + 1]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
template <bool TF32> struct Split;
template <> struct Split<false> {
    using E = __nv_bfloat16;
    __device__ static void run(double x, E &hi, E &lo) {
        hi = __double2bfloat16(x);
        lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    }
};
template <> struct Split<true> {
    using E = float;
    __device__ static float tf32(float x) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return __uint_as_float(r);
    }
    __device__ static void run(double x, E &hi, E &lo) {
        hi = tf32((float)x);
        lo = tf32((float)(x - (double)hi));
    }
};

// A parts from the exact grid phases: [4][Nq][Kp] = (Re hi, Re lo, Im hi, Im lo), zero for p >= nR.
// Row r is grid point pts[r] (pts = null: grid point r); the long-range columns
// (L, nL) belong to the q table only.
template <bool TF32>
__global__ void k_split_phases(int n1, int n2, int n3, int64_t Nq, const int32_t *__restrict__ pts,
                               const int32_t *__restrict__ R, int nR, int Kp,
                               typename Split<TF32>::E *__restrict__ out, const double2 *__restrict__ L, int nL) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Nq * Kp) return;
    const int64_t row = t / Kp;
    const int64_t q = pts ? (int64_t)pts[row] : row;
    const int p = (int)(t % Kp);
    double c = 0.0, s = 0.0;
    if (p >= nR && p < nR + nL) {   // long-range columns (polar coupling)
        const double2 v = L[row * nL + (p - nR)];
        c = v.x;
        s = v.y;
    } else if (p < nR) {
        const int i3 = (int)(q % n3), i2 = (int)((q / n3) % n2), i1 = (int)(q / ((int64_t)n2 * n3));
        int t1 = (int)(((int64_t)i1 * R[3 * p + 0]) % n1);
        int t2 = (int)(((int64_t)i2 * R[3 * p + 1]) % n2);
        int t3 = (int)(((int64_t)i3 * R[3 * p + 2]) % n3);
        if (t1 < 0) t1 += n1;
        if (t2 < 0) t2 += n2;
        if (t3 < 0) t3 += n3;
        double x = (double)t1 / n1 + (double)t2 / n2 + (double)t3 / n3;
        x -= rint(x);
        sincospi(2.0 * x, &s, &c);
    }
    typename Split<TF32>::E h, l;
    const int64_t part = Nq * Kp;
    Split<TF32>::run(c, h, l);
    out[0 * part + t] = h;
    out[1 * part + t] = l;
    Split<TF32>::run(s, h, l);
    out[2 * part + t] = h;
    out[3 * part + t] = l;
}

// A parts from a complex FP64 table of arbitrary points (phases e^{i k.R} of
// off-grid k or q, with any long-range columns appended): T[r][p] for r < n,
// p < ncols (row stride ld) -> [4][n][Kp] = (Re hi, Re lo, Im hi, Im lo), zero
// for p >= ncols.
template <bool TF32>
__global__ void k_split_table(int64_t n, int ncols, int64_t ld, int Kp, const double2 *__restrict__ T,
                              typename Split<TF32>::E *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t part = n * Kp;
    if (t >= part) return;
    const int64_t r = t / Kp;
    const int p = (int)(t % Kp);
    const double2 v = p < ncols ? T[r * ld + p] : make_double2(0.0, 0.0);
    typename Split<TF32>::E h, l;
    Split<TF32>::run(v.x, h, l);
    out[0 * part + t] = h;
    out[1 * part + t] = l;
    Split<TF32>::run(v.y, h, l);
    out[2 * part + t] = h;
    out[3 * part + t] = l;
}

// B parts of one k-batch: G[b][p][c] (FP32 complex, ncol_in columns) -> [b][4][ncol][Kp],
// zero in the padding columns c >= ncol_in.
template <bool TF32>
__global__ void k_split_g(int64_t nb, int nR, int ncol_in, int ncol, int Kp, const float2 *__restrict__ G,
                          typename Split<TF32>::E *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)ncol * Kp;
    if (t >= nb * per) return;
    const int64_t b = t / per;
    const int64_t r = t % per;
    const int c = (int)(r / Kp);
    const int p = (int)(r % Kp);
    float2 v = make_float2(0.f, 0.f);
    if (p < nR && c < ncol_in) v = G[(b * nR + p) * ncol_in + c];
    typename Split<TF32>::E h, l;
    typename Split<TF32>::E *o = out + b * 4 * per + r;
    Split<TF32>::run((double)v.x, h, l);
    o[0 * per] = h;
    o[1 * per] = l;
    Split<TF32>::run((double)v.y, h, l);
    o[2 * per] = h;
    o[3 * per] = l;
}

// B parts for the fused kernel: [b][6][ncol][Kp] = Br_hi, Br_lo, Bi_hi, Bi_lo,
// -Bi_hi, -Bi_lo (the negated copy lets one MMA form [C_re | C_im]).
template <bool TF32>
__global__ void k_split_g6(int64_t nb, int nR, int ncol, int Kp, const float2 *__restrict__ G,
                           typename Split<TF32>::E *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)ncol * Kp;
    if (t >= nb * per) return;
    const int64_t b = t / per;
    const int64_t r = t % per;
    const int c = (int)(r / Kp);
    const int p = (int)(r % Kp);
    float2 v = make_float2(0.f, 0.f);
    if (p < nR) v = G[(b * nR + p) * ncol + c];
    typename Split<TF32>::E h, l;
    typename Split<TF32>::E *o = out + b * 6 * per + r;
    Split<TF32>::run((double)v.x, h, l);
    o[0 * per] = h;
    o[1 * per] = l;
    Split<TF32>::run((double)v.y, h, l);
    o[2 * per] = h;
    o[3 * per] = l;
    o[4 * per] = -h;
    o[5 * per] = -l;
}

// B parts of the R_e sum (Eq. eph_mat_wann2, first factor): g~[p][c] (p < nR = R_e,
// c < ncol = R_p x modes x bands^2) -> [4][ncol][Kp] = (re hi, re lo, im hi, im lo),
// K = R_e fastest, zero for p >= nR.
template <bool TF32>
__global__ void k_split_gT(int nR, int64_t ncol, int Kp, const double2 *__restrict__ g,
                           typename Split<TF32>::E *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = ncol * Kp;
    if (t >= per) return;
    const int64_t c = t / Kp;
    const int p = (int)(t % Kp);
    double2 v = make_double2(0.0, 0.0);
    if (p < nR) v = g[(int64_t)p * ncol + c];
    typename Split<TF32>::E h, l;
    Split<TF32>::run(v.x, h, l);
    out[0 * per + t] = h;
    out[1 * per + t] = l;
    Split<TF32>::run(v.y, h, l);
    out[2 * per + t] = h;
    out[3 * per + t] = l;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map over [d2][d1][Kp] with a box of EK x rows x 1 and the 64-byte swizzle.
// Returns the driver's CUresult (-1 if the encoder could not be loaded).
int make_map(CUtensorMap *m, void *base, bool tf32, int Kp, int64_t d1, int64_t d2, int box_rows) {
    auto enc = encode_fn();
    if (!enc) return -1;
    const int esz = tf32 ? 4 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)d1, (cuuint64_t)d2};
    const cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)Kp * esz * d1};
    const cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (int)r;
}

// One thread waits on an mbarrier that nothing arrives on, with the same
// bounded wait the pipelines use; the run-out is reported through *err.
__global__ void k_wait_timeout(long long budget, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_addr(&bar), 1);
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(tc::smem_addr(&bar), 0, budget)) atomicOr(err, 8);
}

}  // namespace

int tc_kpad(int nR) { return ((nR + 31) / 32) * 32; }

bool tc_supported(int ncol) { return ncol % BN == 0; }

pgb_status launch_split_phases(pgb_ctx *c, bool tf32, const int grid[3], int64_t Nq, const int32_t *d_R, int nR,
                               int Kp, void *out, const double2 *L, int nL) {
    const int64_t n = Nq * Kp;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (!L) nL = 0;
    if (tf32)
        k_split_phases<true><<<g, 256, 0, c->stream>>>(grid[0], grid[1], grid[2], Nq, nullptr, d_R, nR, Kp,
                                                       (float *)out, L, nL);
    else
        k_split_phases<false><<<g, 256, 0, c->stream>>>(grid[0], grid[1], grid[2], Nq, nullptr, d_R, nR, Kp,
                                                        (__nv_bfloat16 *)out, L, nL);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_split_phases_pts(pgb_ctx *c, bool tf32, const int grid[3], const int32_t *d_pts, int64_t n,
                                   const int32_t *d_R, int nR, int Kp, void *out) {
    if (n == 0) return PGB_OK;
    const unsigned g = (unsigned)((n * Kp + 255) / 256);
    if (tf32)
        k_split_phases<true><<<g, 256, 0, c->stream>>>(grid[0], grid[1], grid[2], n, d_pts, d_R, nR, Kp,
                                                       (float *)out, nullptr, 0);
    else
        k_split_phases<false><<<g, 256, 0, c->stream>>>(grid[0], grid[1], grid[2], n, d_pts, d_R, nR, Kp,
                                                        (__nv_bfloat16 *)out, nullptr, 0);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_split_table(pgb_ctx *c, bool tf32, int64_t n, int ncols, int64_t ld, int Kp, const double2 *T,
                              void *out) {
    const int64_t tot = n * Kp;
    if (tot == 0) return PGB_OK;
    const unsigned g = (unsigned)((tot + 255) / 256);
    if (tf32)
        k_split_table<true><<<g, 256, 0, c->stream>>>(n, ncols, ld, Kp, T, (float *)out);
    else
        k_split_table<false><<<g, 256, 0, c->stream>>>(n, ncols, ld, Kp, T, (__nv_bfloat16 *)out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_split_gT(pgb_ctx *c, bool tf32, int nR, int64_t ncol, int Kp, const double2 *g, void *out) {
    const int64_t n = ncol * Kp;
    const unsigned gr = (unsigned)((n + 255) / 256);
    if (tf32)
        k_split_gT<true><<<gr, 256, 0, c->stream>>>(nR, ncol, Kp, g, (float *)out);
    else
        k_split_gT<false><<<gr, 256, 0, c->stream>>>(nR, ncol, Kp, g, (__nv_bfloat16 *)out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_split_g(pgb_ctx *c, bool tf32, int64_t nb, int nR, int ncol, int Kp, const void *G, void *out,
                          int ncol_pad) {
    const int ncol_out = ncol_pad > ncol ? ncol_pad : ncol;
    const int64_t n = nb * (int64_t)ncol_out * Kp;
    if (n == 0) return PGB_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (tf32)
        k_split_g<true><<<g, 256, 0, c->stream>>>(nb, nR, ncol, ncol_out, Kp, (const float2 *)G, (float *)out);
    else
        k_split_g<false><<<g, 256, 0, c->stream>>>(nb, nR, ncol, ncol_out, Kp, (const float2 *)G,
                                                   (__nv_bfloat16 *)out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_split_g6(pgb_ctx *c, bool tf32, int64_t nb, int nR, int ncol, int Kp, const void *G, void *out) {
    const int64_t n = nb * (int64_t)ncol * Kp;
    if (n == 0) return PGB_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (tf32)
        k_split_g6<true><<<g, 256, 0, c->stream>>>(nb, nR, ncol, Kp, (const float2 *)G, (float *)out);
    else
        k_split_g6<false><<<g, 256, 0, c->stream>>>(nb, nR, ncol, Kp, (const float2 *)G, (__nv_bfloat16 *)out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

// C[b][q][c] for b < nb from the split operands; err (device int) collects
// wait time-outs and is checked by the caller.
pgb_status launch_tc_qsum(pgb_ctx *c, bool tf32, int64_t nb, int64_t Nq, int ncol, int Kp, void *Asplit,
                          void *Bsplit, float2 *C, int *d_err, int64_t nqA, int64_t q_off) {
    if (nb == 0 || Nq == 0) return PGB_OK;
    if (nqA <= 0) nqA = Nq;
    if (q_off < 0 || q_off + Nq > nqA || nqA > INT32_MAX) {
        c->err = "tensor-core q-sum: q rows outside the A table";
        return PGB_EINVAL;
    }
    if (ncol % BN != 0 || Kp % 32 != 0 || nb > 65535 || (Nq + BM - 1) / BM > 65535) {
        c->err = "tensor-core q-sum: unsupported shape (needs nmode*nw*nw a multiple of 96)";
        return PGB_EINVAL;
    }
    CUtensorMap tA, tB;
    const int ra = make_map(&tA, Asplit, tf32, Kp, nqA, 4, BM);
    const int rb = ra == 0 ? make_map(&tB, Bsplit, tf32, Kp, ncol, nb * 4, BN) : 0;
    if (ra != 0 || rb != 0) {
        c->err = "tensor-core q-sum: cuTensorMapEncodeTiled failed (A " + std::to_string(ra) + ", B " +
                 std::to_string(rb) + ")";
        return PGB_ECUDA;
    }
    TcArgs a;
    a.Nq = Nq;
    a.q_off = (int)q_off;
    a.Kp = Kp;
    a.ncol = ncol;
    a.nb = (int)nb;
    a.C = C;
    a.err = d_err;
    dim3 grid((unsigned)(ncol / BN), (unsigned)((Nq + BM - 1) / BM), (unsigned)nb);
    const pgb_status pst = tc_qsum_prepare(c, tf32);
    if (pst != PGB_OK) return pst;
    if (tf32)
        k_tc_qsum_tf32<<<grid, TF_THREADS, SMEM_BYTES, c->stream>>>(tA, tB, a);
    else
        k_tc_qsum<false><<<grid, 192, SMEM_BYTES, c->stream>>>(tA, tB, a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

// Shared-memory limit of k_tc_qsum on the context's device, set once per device and
// form (so that launches under stream capture need no attribute call).
pgb_status tc_qsum_prepare(pgb_ctx *c, bool tf32) {
    static std::mutex mu;
    static std::vector<char> done[2];
    std::lock_guard<std::mutex> lock(mu);
    std::vector<char> &d = done[tf32 ? 1 : 0];
    if (c->device >= 0 && (size_t)c->device < d.size() && d[c->device]) return PGB_OK;
    if (tf32)
        PGB_CUDA_TRY(c, cudaFuncSetAttribute(k_tc_qsum_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    else
        PGB_CUDA_TRY(c, cudaFuncSetAttribute(k_tc_qsum<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    if (c->device >= 0) {
        if ((size_t)c->device >= d.size()) d.resize(c->device + 1, 0);
        d[c->device] = 1;
    }
    return PGB_OK;
}

}  // namespace pgb

// Diagnostic: exercise the bounded-wait path (see include/pertgb_diag.h).
extern "C" pgb_status pgb_selftest_wait_timeout(pgb_ctx *c, long long budget_cycles) {
    using namespace pgb;
    if (!c || budget_cycles <= 0 || budget_cycles > (1ll << 32)) return PGB_EINVAL;
    cudaSetDevice(c->device);
    int *d = nullptr;
    PGB_CUDA_TRY(c, dev_malloc((void **)&d, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        k_wait_timeout<<<1, 32, 0, c->stream>>>(budget_cycles, d);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) {
        c->err = std::string("selftest_wait_timeout: ") + cudaGetErrorString(e);
        return PGB_ECUDA;
    }
    if (h) {
        c->err = "selftest_wait_timeout: the wait ran out as intended (bits " + std::to_string(h) + ")";
        return PGB_ETIMEOUT;
    }
    return PGB_OK;
}
