// Band interpolation at arbitrary points for the FP32 paths: a real form of the
// Fourier sum and a mixed-precision Jacobi eigensolver (Sec. 2.2.1, Eq.
// wannier_3: H(k) = sum_R e^{ik.R} H(R), H(k) = U(k) diag(eps_k) U(k)^dagger).
//
// Fourier sum.  The eigensolver uses the Hermitian part of H(k), which is, for any
// set of R closed under inversion,
//   H(k) = sum_{R in S} cos(k.R) C_R + sin(k.R) S_R,
//   C_R = A(R) + A(-R),  S_R = B(R) - B(-R)   (C_0 = A(0), S_0 = 0),
//   A(X) = (H(X) + H(X)^dagger) / 2,  B(X) = i (H(X) - H(X)^dagger) / 2,
// over one representative R of each pair {R, -R}.  C_R and S_R are Hermitian,
// so only the upper triangle is summed: nw real diagonal entries and the real
// and imaginary parts of the nw (nw - 1) / 2 entries above it, nw^2 real
// columns.  That is a real GEMM with K = 2 |S| ~ nR rows, a quarter of the real
// multiply-adds of the complex form.  The phases come from per-point 1-D tables
// e^{2 pi i k_d m}: e^{ik.R} = prod_d e^{2 pi i k_d R_d}.  The sum runs in
// double-float arithmetic on the FP32 pipe (see k_herm_sum).
//
// Eigensolver.  A parallel cyclic Jacobi with one lane per matrix row: in each
// round the n/2 disjoint pairs of a round-robin schedule are rotated at once
// (columns in every lane, rows by exchanging the two rows of each pair).  The
// rotation is the one of the FP64 thread-per-matrix solver (phase of the pivot
// removed, then the real rotation that zeroes it).  It runs
//   1. in FP32 with eigenvectors, to convergence at FP32 rounding (V);
//   2. in FP64 without eigenvectors on A'' below, for the eigenvalues:
//        A' = V^dagger H V,  E = V^dagger V - I   (both in double-float),
//        A''_ij = A'_ij - E_ij (A'_ii + A'_jj) / 2,
//      the congruence of A' by (I + E)^{-1/2} (symmetric orthonormalisation of
//      V) to first order in E; the terms left out are O(|E|^2 |H|) and
//      O(|E| |A'_ij, i != j|), below 1e-11 of |H| for |E| ~ 1e-7.  A'' is nearly
//      diagonal (off-diagonals ~1e-7 |H|): where every coupling is below 1e-4 of
//      its gap, second-order perturbation theory gives the eigenvalues (see the
//      kernel); otherwise one sweep, quadratically convergent, leaves couplings
//      b ~ 1e-12 |H| or below, which move an eigenvalue by at most
//      min(|b|, |b|^2 / gap).  The sweeps stop once the off-diagonal mass is
//      below 1e-22 of the total.
// The eigenvalues are those of H to FP64 rounding; the eigenvectors returned are
// the FP32 V (orthonormal to ~1e-7), which is what the FP32 |g|^2 products use.
// Within a cluster of eigenvalues closer than ~1e-7 |H| the FP32 vectors are an
// orthonormal basis of the cluster's subspace in an arbitrary gauge, as at an
// exact degeneracy: sums over the bands of a cluster are unaffected.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "herm_table.h"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

constexpr int kHermMaxM = 7;      // per-point 1-D phase tables for |R_d| <= 7, else one sincospi per (point, R)
constexpr int HS_P = 64;          // points per block of the Fourier sum
constexpr int HS_C = 64;          // real columns per block
constexpr int HS_K = 16;          // K rows (8 representatives) per stage

// Double-float arithmetic on the FP32 pipe (a value is an unevaluated sum h + l of
// two floats, ~48 significant bits).  Every step uses the explicitly rounded
// intrinsics so that the compiler cannot contract a product and a sum into an FMA
// (the error-free transforms below depend on each rounding).
__device__ __forceinline__ float2 df_split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
// h + l = a + b exactly, |l| <= ulp(h)/2, for |a| >= |b| or a = 0
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float h = __fadd_rn(a, b);
    return make_float2(h, __fsub_rn(b, __fsub_rn(h, a)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float z = __fsub_rn(s, a.x);
    float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z));
    t = __fadd_rn(t, __fadd_rn(a.y, b.y));
    return fast_two_sum(s, t);
}
struct cdf {   // complex double-float
    float2 re, im;
};
__device__ __forceinline__ cdf cdf_mul(const cdf &x, const cdf &y) {
    cdf r;
    const float2 a = df_mul(x.re, y.re), b = df_mul(x.im, y.im), c = df_mul(x.re, y.im), d = df_mul(x.im, y.re);
    r.re = df_add(a, make_float2(-b.x, -b.y));
    r.im = df_add(c, d);
    return r;
}
// (sh, sl) += (ah + al)(bh + bl): exact leading product and its error, TwoSum into sh;
// the al bl term (2^-48 relative) is dropped
__device__ __forceinline__ void df_fma(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float r = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(r, e));
    sh = t;
}

// (sh, sl) += (xh + xl) y: the product exact to ~2^-48, TwoSum into sh
__device__ __forceinline__ void df_acc_mulf(float &sh, float &sl, float2 x, float y) {
    const float p = __fmul_rn(x.x, y);
    float e = __fmaf_rn(x.x, y, -p);
    e = __fmaf_rn(x.y, y, e);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float r = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(r, e));
    sh = t;
}
// (sh, sl) += x y for floats: the product exact as p + e
__device__ __forceinline__ void df_acc_ff(float &sh, float &sl, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float r = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(r, e));
    sh = t;
}
__device__ __forceinline__ void df_renorm(float &sh, float &sl) {
    const float2 n = fast_two_sum(sh, sl);
    sh = n.x;
    sl = n.y;
}

// Real Fourier sum: out[p][c] = sum_k phase_k(p) T[k][c], phase_{2r} = cos(2 pi k.R_r),
// phase_{2r+1} = sin(2 pi k.R_r), in double-float (products and sums on the FP32
// pipe, ~2^-44 relative to the largest partial sum; FP64 would be FP64-pipe bound).
// Block: 64 points x 64 columns, 4 x 4 per thread.  The phases are products of
// per-point 1-D tables e^{2 pi i k_d m} (powers of sincospi(2 k_d) in
// double-float) when every |R_d| <= kHermMaxM, else one FP64 sincospi each.
__global__ void __launch_bounds__(256) k_herm_sum(int64_t np, const double *__restrict__ pts, int nrep,
                                                  const int32_t *__restrict__ Rrep, int M, int ncol,
                                                  const float2 *__restrict__ T2, double *__restrict__ out) {
    extern __shared__ float4 t1d[];   // [3][2M+1][HS_P] (re_h, re_l, im_h, im_l), when M <= kHermMaxM
    __shared__ __align__(16) float Ah[HS_K][HS_P];
    __shared__ __align__(16) float Al[HS_K][HS_P];
    __shared__ __align__(16) float Bh[HS_K][HS_C];
    __shared__ __align__(16) float Bl[HS_K][HS_C];
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * HS_P;
    const int c0 = blockIdx.y * HS_C;
    const int W = 2 * M + 1;
    const bool tab = M <= kHermMaxM;
    if (tab) {
        for (int x = tid; x < 3 * HS_P; x += blockDim.x) {
            const int pl = x % HS_P, d = x / HS_P;
            const int64_t p = p0 + pl;
            double sn = 0.0, cs = 1.0;
            if (p < np) sincospi(2.0 * pts[3 * p + d], &sn, &cs);
            cdf b, pw;
            b.re = df_split(cs);
            b.im = df_split(sn);
            pw.re = make_float2(1.f, 0.f);
            pw.im = make_float2(0.f, 0.f);
            float4 *row = t1d + (size_t)d * W * HS_P + pl;
            row[M * HS_P] = make_float4(1.f, 0.f, 0.f, 0.f);
            for (int m = 1; m <= M; ++m) {
                pw = cdf_mul(pw, b);
                row[(M + m) * HS_P] = make_float4(pw.re.x, pw.re.y, pw.im.x, pw.im.y);
                row[(M - m) * HS_P] = make_float4(pw.re.x, pw.re.y, -pw.im.x, -pw.im.y);
            }
        }
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
    const int K = 2 * nrep;
    for (int k0 = 0; k0 < K; k0 += HS_K) {
        for (int x = tid; x < (HS_K / 2) * HS_P; x += blockDim.x) {
            const int pl = x % HS_P, rl = x / HS_P;
            const int rep = k0 / 2 + rl;
            const int64_t p = p0 + pl;
            cdf e;
            e.re = e.im = make_float2(0.f, 0.f);
            if (rep < nrep && p < np) {
                const int R1 = Rrep[3 * rep], R2 = Rrep[3 * rep + 1], R3 = Rrep[3 * rep + 2];
                if (tab) {
                    const float4 f1 = t1d[(R1 + M) * HS_P + pl], f2 = t1d[(W + R2 + M) * HS_P + pl],
                                 f3 = t1d[(2 * W + R3 + M) * HS_P + pl];
                    cdf a1, a2, a3;
                    a1.re = make_float2(f1.x, f1.y), a1.im = make_float2(f1.z, f1.w);
                    a2.re = make_float2(f2.x, f2.y), a2.im = make_float2(f2.z, f2.w);
                    a3.re = make_float2(f3.x, f3.y), a3.im = make_float2(f3.z, f3.w);
                    e = cdf_mul(cdf_mul(a1, a2), a3);
                } else {
                    double x3 = pts[3 * p] * R1 + pts[3 * p + 1] * R2 + pts[3 * p + 2] * R3;
                    x3 -= rint(x3);
                    double sn, cs;
                    sincospi(2.0 * x3, &sn, &cs);
                    e.re = df_split(cs);
                    e.im = df_split(sn);
                }
            }
            Ah[2 * rl][pl] = e.re.x;
            Al[2 * rl][pl] = e.re.y;
            Ah[2 * rl + 1][pl] = e.im.x;
            Al[2 * rl + 1][pl] = e.im.y;
        }
        for (int x = tid; x < HS_K * HS_C; x += blockDim.x) {
            const int cl = x % HS_C, kl = x / HS_C;
            const int kr = k0 + kl, col = c0 + cl;
            const float2 v = (kr < K && col < ncol) ? T2[(int64_t)kr * ncol + col] : make_float2(0.f, 0.f);
            Bh[kl][cl] = v.x;
            Bl[kl][cl] = v.y;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < HS_K; ++kk) {
            const float4 ah = *reinterpret_cast<const float4 *>(&Ah[kk][ty * 4]);
            const float4 al = *reinterpret_cast<const float4 *>(&Al[kk][ty * 4]);
            const float4 bh = *reinterpret_cast<const float4 *>(&Bh[kk][tx * 4]);
            const float4 bl = *reinterpret_cast<const float4 *>(&Bl[kk][tx * 4]);
            const float ahv[4] = {ah.x, ah.y, ah.z, ah.w}, alv[4] = {al.x, al.y, al.z, al.w};
            const float bhv[4] = {bh.x, bh.y, bh.z, bh.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) df_fma(sh[i][j], sl[i][j], ahv[i], alv[i], bhv[j], blv[j]);
            if (kk & 1) {   // renormalise every second step: |sl| stays near ulp(sh)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float2 n = fast_two_sum(sh[i][j], sl[i][j]);
                        sh[i][j] = n.x;
                        sl[i][j] = n.y;
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t p = p0 + ty * 4 + i;
        if (p >= np) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = c0 + tx * 4 + j;
            if (col < ncol) out[p * ncol + col] = (double)sh[i][j] + (double)sl[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// Parallel Jacobi, one lane per row
// ---------------------------------------------------------------------------
template <int N>
struct JShape {
    static constexpr int L = N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16;   // lanes per matrix (one per row)
    static constexpr int NE = N + (N & 1);   // indices of the round-robin schedule (one dummy when N is odd)
    static constexpr int NR = NE - 1;        // rounds per sweep
    static constexpr int NP = NE / 2;        // pairs per round
};

// Circle schedule over ne indices: in round t index ne-1 meets t, and t+k meets
// t-k (mod ne-1) for k = 1 .. ne/2-1.  Partner of index r in round t:
__device__ __forceinline__ int rr_partner(int ne, int t, int r) {
    const int m = ne - 1;
    if (r == m) return t;
    if (r == t) return m;
    const int x = (2 * t - r) % m;
    return x < 0 ? x + m : x;
}

template <typename T2, int N>
__device__ __forceinline__ T2 pick(const T2 (&a)[N], int idx) {
    T2 v = a[0];
#pragma unroll
    for (int e = 1; e < N; ++e)
        if (e == idx) v = a[e];
    return v;
}

// Rotation that zeroes the pivot b = A_pq of the Hermitian 2x2 block
// [[app, b], [conj b, aqq]]: with e = conj(b)/|b|, z = (aqq - app) / (2|b|),
// t = sgn(z) / (|z| + sqrt(z^2 + 1)), c = 1/sqrt(1 + t^2), s = t c, the
// columns (p, q) of J are (c, -s e) and (s, c e).  Returns the identity for b = 0.
// |b| and e are formed from b scaled by max(|Re b|, |Im b|): inside a degenerate
// cluster the pivots become tiny, and an unscaled |b|^2 would underflow and
// leave |e| != 1 (J no longer unitary).  Pivots below 1e-30 (where 1/max could
// overflow in FP32) are left to the exact zeroing that follows every rotation,
// which moves the eigenvalues by at most |b|.
template <typename T>
__device__ __forceinline__ void rot_params(T app, T aqq, T br, T bi, T &c, T &s, T &pr, T &pi, T &qr, T &qi) {
    const T mx = fmax(fabs(br), fabs(bi));
    if (!(mx > T(1e-30))) return;
    const T im = T(1) / mx;
    const T xr = br * im, xi = bi * im;
    const T nn = sqrt(xr * xr + xi * xi);
    const T inn = T(1) / nn;
    const T er = xr * inn, ei = -xi * inn;
    const T ab = mx * nn;
    const T z = (aqq - app) / (T(2) * ab);
    T t;
    if (fabs(z) > T(1e18))
        t = T(0.5) / z;
    else
        t = (z >= T(0) ? T(1) : T(-1)) / (fabs(z) + sqrt(z * z + T(1)));
    c = T(1) / sqrt(T(1) + t * t);
    s = t * c;
    pr = -s * er;
    pi = -s * ei;
    qr = c * er;
    qi = c * ei;
}

// FP64 form for the eigenvalue stage (pivots far above underflow there): rsqrt and a
// correctly rounded reciprocal instead of divides; c^2 + s^2 = 1 and |e| = 1 to a
// few ulp, so J stays unitary to FP64 rounding.  A pivot below 1e-140 is left to
// the exact zeroing that follows every rotation (its effect on the eigenvalues is
// below |b|^2 / gap).
__device__ __forceinline__ void rot_params64(double app, double aqq, double br, double bi, double &c, double &s,
                                             double &pr, double &pi, double &qr, double &qi) {
    const double b2 = fma(br, br, bi * bi);
    if (!(b2 > 1e-280)) return;
    const double inv = rsqrt(b2);
    const double er = br * inv, ei = -bi * inv;
    const double z = (aqq - app) * (0.5 * inv);
    const double az = fabs(z);
    double t;
    if (az > 1e18) {
        t = __drcp_rn(2.0 * z);
    } else {
        const double z2 = fma(z, z, 1.0);
        const double rt = z2 * rsqrt(z2);
        t = copysign(__drcp_rn(az + rt), z);
    }
    c = rsqrt(fma(t, t, 1.0));
    s = t * c;
    pr = -s * er;
    pi = -s * ei;
    qr = c * er;
    qi = c * ei;
}

// (x, y) <- (c x + vp y, s x + vq y): entries p, q of one row of A J
template <typename T2, typename T>
__device__ __forceinline__ void rot_cols(T2 &x, T2 &y, T c, T s, T pr, T pi, T qr, T qi) {
    const T2 x0 = x, y0 = y;
    x.x = c * x0.x + (pr * y0.x - pi * y0.y);
    x.y = c * x0.y + (pr * y0.y + pi * y0.x);
    y.x = s * x0.x + (qr * y0.x - qi * y0.y);
    y.y = s * x0.y + (qr * y0.y + qi * y0.x);
}

// Sweeps of the parallel Jacobi on the N x N Hermitian matrix whose row r lane r
// holds in a (lanes base .. base + L - 1 hold one matrix; lanes r >= N hold
// zeros).  With VEC the rows of V (initially I) are rotated too, so that
// A_in = V A_out V^dagger.  Stops when every matrix of the warp has
// sum_{i != j} |A_ij|^2 <= tol * sum |A_ij|^2, or after max_sweeps.
template <typename T, int N, bool VEC>
__device__ __forceinline__ void jacobi_rows(V2<T> (&a)[N], V2<T> (&v)[N], int r, int base, T tol,
                                            int max_sweeps) {
    using S = JShape<N>;
    using T2 = V2<T>;
    constexpr unsigned FULL = 0xffffffffu;
    const bool row = r < N;
#pragma unroll 1
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        T off = T(0), tot = T(0);
#pragma unroll
        for (int e = 0; e < N; ++e) {
            const T w = a[e].x * a[e].x + a[e].y * a[e].y;
            tot += w;
            if (e != r) off += w;
        }
#pragma unroll
        for (int o = 1; o < S::L; o <<= 1) {
            off += __shfl_xor_sync(FULL, off, o);
            tot += __shfl_xor_sync(FULL, tot, o);
        }
        if (__all_sync(FULL, !(off > tol * tot))) break;
#pragma unroll
        for (int t = 0; t < S::NR; ++t) {
            const int pt = row ? rr_partner(S::NE, t, r) : r;
            const bool paired = row && pt < N;
            const int src = base + (paired ? pt : r);
            // pivots of this lane's pair: lane p holds A_pp and A_pq, lane q holds A_qq
            const T dg = pick(a, r).x;
            const T2 of = pick(a, pt);
            const T dg_o = __shfl_sync(FULL, dg, src);
            const T ofx_o = __shfl_sync(FULL, of.x, src), ofy_o = __shfl_sync(FULL, of.y, src);
            const bool is_p = r < pt;
            T c = T(1), s = T(0), pr = T(0), pi = T(0), qr = T(1), qi = T(0);
            if (paired) {
                if constexpr (sizeof(T) == 8)
                    rot_params64(is_p ? dg : dg_o, is_p ? dg_o : dg, is_p ? of.x : ofx_o, is_p ? of.y : ofy_o, c, s,
                                 pr, pi, qr, qi);
                else
                    rot_params<T>(is_p ? dg : dg_o, is_p ? dg_o : dg, is_p ? of.x : ofx_o, is_p ? of.y : ofy_o, c,
                                  s, pr, pi, qr, qi);
            }
            // A <- A J (and V <- V J): every lane rotates the column pairs of its row
#pragma unroll
            for (int k = 0; k < S::NP; ++k) {
                const int ia = k == 0 ? S::NE - 1 : (t + k) % S::NR;
                const int ib = k == 0 ? t : (t - k + S::NR) % S::NR;
                const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
                if (q >= N) continue;
                const int lp = base + p;
                const T kc = __shfl_sync(FULL, c, lp), ks = __shfl_sync(FULL, s, lp);
                const T kpr = __shfl_sync(FULL, pr, lp), kpi = __shfl_sync(FULL, pi, lp);
                const T kqr = __shfl_sync(FULL, qr, lp), kqi = __shfl_sync(FULL, qi, lp);
                rot_cols(a[p], a[q], kc, ks, kpr, kpi, kqr, kqi);
                if (VEC) rot_cols(v[p], v[q], kc, ks, kpr, kpi, kqr, kqi);
            }
            // A <- J^dagger A: row p' = c row p + conj(vp) row q, row q' = s row p + conj(vq) row q,
            // i.e. new row = ar X + conj(b) Y with (ar, b, X, Y) = (c, vp, own, partner) in lane p
            // and (s, vq, partner, own) in lane q: one real and one complex coefficient
            T ar = T(1), bx = T(0), by = T(0);
            if (paired) {
                ar = is_p ? c : s;
                bx = is_p ? pr : qr;
                by = is_p ? pi : qi;
            }
            const bool swap = paired && !is_p;
#pragma unroll
            for (int e = 0; e < N; ++e) {
                T2 o;
                o.x = __shfl_sync(FULL, a[e].x, src);
                o.y = __shfl_sync(FULL, a[e].y, src);
                const T2 X = swap ? o : a[e], Y = swap ? a[e] : o;
                a[e].x = fma(ar, X.x, fma(bx, Y.x, by * Y.y));
                a[e].y = fma(ar, X.y, fma(bx, Y.y, -(by * Y.x)));
            }
            // the rotated pivots are zero and the diagonal real, exactly
#pragma unroll
            for (int k = 0; k < S::NP; ++k) {
                const int ia = k == 0 ? S::NE - 1 : (t + k) % S::NR;
                const int ib = k == 0 ? t : (t - k + S::NR) % S::NR;
                const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
                if (q >= N) continue;
                if (r == p) {
                    a[q].x = T(0);
                    a[q].y = T(0);
                    a[p].y = T(0);
                }
                if (r == q) {
                    a[p].x = T(0);
                    a[p].y = T(0);
                    a[q].y = T(0);
                }
            }
        }
    }
}

// entry (r, l) of the Hermitian matrix from its packed upper triangle
// (diagonal reals first, then (re, im) of (i, j), i < j, row by row)
template <int N>
__device__ __forceinline__ double2 packed_entry(const double *__restrict__ H, int r, int l) {
    if (l == r) return make_double2(H[r], 0.0);
    const int i = r < l ? r : l, j = r < l ? l : r;
    const int idx = N + 2 * (i * N - (i * (i + 1)) / 2 + (j - i - 1));
    return make_double2(H[idx], r < l ? H[idx + 1] : -H[idx + 1]);
}

// Eigenpairs of count packed Hermitian N x N matrices: eigenvalues ascending
// (FP64-refined), eigenvector columns in U[i][n] order: the FP32 V, or with VREF
// refined in FP64 as well, U = V (I - E/2) J with J the FP64 rotations (the
// orthonormalised basis times the eigenvectors of A'').  VREF serves the phonon
// modes: near q = 0 the acoustic omega^2 are ~1e-6 of |D| apart, below what the
// FP32 vectors resolve, and the mode coefficients sqrt(hbar / 2 M omega) differ
// between those branches.
template <int N, bool VREF>
__global__ void __launch_bounds__(64) k_heev_mixed(int64_t count, const double *__restrict__ Hp,
                                                   double *__restrict__ eval, float2 *__restrict__ U32,
                                                   double2 *__restrict__ U64) {
    using S = JShape<N>;
    constexpr int MPB = 64 / S::L;   // matrices per block
    constexpr int NC = N * N;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ float2 Vs[MPB][N][N];
    __shared__ double2 Ws[MPB][N][N];
    const int lane = threadIdx.x & 31;
    const int r = lane & (S::L - 1), base = lane & ~(S::L - 1);
    const int ms = threadIdx.x / S::L;
    const int64_t pt = (int64_t)blockIdx.x * MPB + ms;
    const bool row = r < N;
    const bool live = row && pt < count;
    const int rc = row ? r : 0;
    const double *H = Hp + (pt < count ? pt : 0) * (int64_t)NC;
    // 1. FP32 Jacobi with eigenvectors
    float2 a[N], v[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
        const double2 x = live ? packed_entry<N>(H, r, l) : make_double2(0.0, 0.0);
        a[l] = make_float2((float)x.x, (float)x.y);
        v[l] = make_float2(live && l == r ? 1.f : 0.f, 0.f);
    }
    jacobi_rows<float, N, true>(a, v, r, base, 1e-12f, 15);
    if (row) {
#pragma unroll
        for (int e = 0; e < N; ++e) Vs[ms][r][e] = v[e];
    }
    __syncwarp();
    // 2. W = H V (row r) in double-float: H split into (hi, lo) floats, V exact
    //    floats; each product exact to ~2^-48, TwoSum accumulation renormalised
    //    every fourth term (the FP64 form of stages 2-3 was most of the FP64 work)
    {
        float4 *Wd = reinterpret_cast<float4 *>(&Ws[ms][0][0]);
        float wrh[N], wrl[N], wih[N], wil[N];
#pragma unroll
        for (int j = 0; j < N; ++j) wrh[j] = wrl[j] = wih[j] = wil[j] = 0.f;
#pragma unroll 1
        for (int l = 0; l < N; ++l) {   // outer loops rolled: the unrolled body overflowed the instruction cache
            const double2 h = live ? packed_entry<N>(H, r, l) : make_double2(0.0, 0.0);
            const float2 hr = df_split(h.x), hi = df_split(h.y);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float2 vl = Vs[ms][l][j];
                df_acc_mulf(wrh[j], wrl[j], hr, vl.x);   // re = hr vx - hi vy
                df_acc_mulf(wrh[j], wrl[j], hi, -vl.y);
                df_acc_mulf(wih[j], wil[j], hr, vl.y);   // im = hr vy + hi vx
                df_acc_mulf(wih[j], wil[j], hi, vl.x);
            }
            if ((l & 3) == 3) {
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    df_renorm(wrh[j], wrl[j]);
                    df_renorm(wih[j], wil[j]);
                }
            }
        }
        if (row) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                df_renorm(wrh[j], wrl[j]);
                df_renorm(wih[j], wil[j]);
                Wd[r * N + j] = make_float4(wrh[j], wrl[j], wih[j], wil[j]);
            }
        }
    }
    __syncwarp();
    // 3. A' = V^dagger W and E = V^dagger V - I (row r) in double-float, then A''
    //    (first-order congruence) in FP64
    double2 a64[N], v64[N];
    {
        double2 ap[N], ee[N];
        {
            const float4 *Wd = reinterpret_cast<const float4 *>(&Ws[ms][0][0]);
            float arh[N], arl[N], aih[N], ail[N], erh[N], erl[N], eih[N], eil[N];
#pragma unroll
            for (int j = 0; j < N; ++j) arh[j] = arl[j] = aih[j] = ail[j] = erh[j] = erl[j] = eih[j] = eil[j] = 0.f;
#pragma unroll 1
            for (int s = 0; s < N; ++s) {
                const float2 v = Vs[ms][s][rc];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const float4 w = Wd[s * N + j];
                    const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
                    df_acc_mulf(arh[j], arl[j], wr, v.x);    // conj(v) w: re = vx wr + vy wi
                    df_acc_mulf(arh[j], arl[j], wi, v.y);
                    df_acc_mulf(aih[j], ail[j], wi, v.x);    //            im = vx wi - vy wr
                    df_acc_mulf(aih[j], ail[j], wr, -v.y);
                    const float2 vj = Vs[ms][s][j];
                    df_acc_ff(erh[j], erl[j], v.x, vj.x);    // conj(v) vj, products exact
                    df_acc_ff(erh[j], erl[j], v.y, vj.y);
                    df_acc_ff(eih[j], eil[j], v.x, vj.y);
                    df_acc_ff(eih[j], eil[j], -v.y, vj.x);
                }
                if ((s & 3) == 3) {
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        df_renorm(arh[j], arl[j]);
                        df_renorm(aih[j], ail[j]);
                        df_renorm(erh[j], erl[j]);
                        df_renorm(eih[j], eil[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                ap[j] = make_double2((double)arh[j] + (double)arl[j], (double)aih[j] + (double)ail[j]);
                ee[j] = make_double2((double)erh[j] + (double)erl[j], (double)eih[j] + (double)eil[j]);
            }
        }
        double lam = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j == r) {
                ee[j].x -= 1.0;
                lam = ap[j].x;
            }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double lj = __shfl_sync(FULL, lam, base + j);
            const double f = 0.5 * (lam + lj);
            a64[j] = live ? make_double2(ap[j].x - f * ee[j].x, ap[j].y - f * ee[j].y) : make_double2(0.0, 0.0);
        }
        if (VREF) {   // row r of V (I - E/2), E from every lane's row
            __syncwarp();
            if (row) {
#pragma unroll
                for (int j = 0; j < N; ++j) Ws[ms][r][j] = ee[j];
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float2 vj = Vs[ms][rc][j];
                v64[j] = make_double2(vj.x, vj.y);
            }
#pragma unroll
            for (int l = 0; l < N; ++l) {
                const float2 vl = Vs[ms][rc][l];
                const double2 h = make_double2(-0.5 * vl.x, -0.5 * vl.y);
#pragma unroll
                for (int j = 0; j < N; ++j) cfma(v64[j], h, Ws[ms][l][j]);
            }
            if (!live) {
#pragma unroll
                for (int j = 0; j < N; ++j) v64[j] = make_double2(0.0, 0.0);
            }
        }
    }
    // 4. Eigenvalues of A''.  Without VREF, when every coupling is small against its
    // gap (|a_ij| <= 1e-4 |a_ii - a_jj| and <= 1e-5 max|a_jj| for all pairs of the
    // warp's matrices), second-order perturbation theory:
    //   lambda_i = a_ii + sum_{j != i} |a_ij|^2 / (a_ii - a_jj),
    // whose third-order remainder is at most (N-1)^2 1e-8 max|a_ij| < 5e-12 of
    // max|a_jj|.  Otherwise (near-degenerate pairs) FP64 Jacobi sweeps on A''.
    bool fast = false;
    double lam_pt = 0.0;
    if constexpr (!VREF) {
        const double dr = pick(a64, r).x;
        double sc = fabs(dr);
#pragma unroll
        for (int o = 1; o < S::L; o <<= 1) sc = fmax(sc, __shfl_xor_sync(FULL, sc, o));
        bool ok = true;
        double corr = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double dj = __shfl_sync(FULL, dr, base + j);
            if (j == r) continue;
            const double gap = dr - dj;
            const double a2 = fma(a64[j].x, a64[j].x, a64[j].y * a64[j].y);
            ok = ok && a2 <= 1e-8 * gap * gap && a2 <= 1e-10 * sc * sc;
            if (a2 > 0.0) corr = fma(a2, __drcp_rn(gap), corr);
        }
        fast = __all_sync(FULL, ok || !live);
        lam_pt = dr + corr;
    }
    if (!fast) jacobi_rows<double, N, VREF>(a64, v64, r, base, 1e-22, 20);
    const double lam = fast ? lam_pt : pick(a64, r).x;
    int rank = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const double lj = __shfl_sync(FULL, lam, base + j);
        rank += (lj < lam || (lj == lam && j < r)) ? 1 : 0;
    }
    if (live) eval[pt * N + rank] = lam;
    if (VREF) {   // lane r holds row r of U: column j goes to position rank_j
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int rj = __shfl_sync(FULL, rank, base + j);
            if (live) {
                if (U32) U32[pt * NC + r * N + rj] = make_float2((float)v64[j].x, (float)v64[j].y);
                if (U64) U64[pt * NC + r * N + rj] = v64[j];
            }
        }
    } else if (live) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float2 u = Vs[ms][i][r];
            if (U32) U32[pt * NC + i * N + rank] = u;
            if (U64) U64[pt * NC + i * N + rank] = make_double2(u.x, u.y);
        }
    }
}

}  // namespace

// Cos/sin coefficient table of X(k) = sum_R e^{ik.R} X(R) (X = H or the mass-scaled
// D; herm_table.h builds it on the host), uploaded when the model is set together
// with its split into (hi, lo) floats for the double-float sum.  X is complex
// [nR][n][n], interleaved (re, im).
pgb_status build_herm_table(pgb_ctx *c, HermTab *tab, const int32_t *R, const double *H, int nR, int nw) {
    std::vector<int32_t> reps;
    std::vector<double> T;
    int M = 0;
    if (!herm_table_host(R, H, nR, nw, reps, T, M)) {
        c->err = "set_model: an R list is not closed under inversion";
        return PGB_EINVAL;
    }
    std::vector<float> T2(2 * T.size());
    for (size_t x = 0; x < T.size(); ++x) {
        const float h = (float)T[x];
        T2[2 * x] = h;
        T2[2 * x + 1] = (float)(T[x] - (double)h);
    }
    pgb_status st = dalloc(c, &tab->d_R, reps.size());
    if (st == PGB_OK) st = dalloc(c, &tab->d_T, T.size());
    if (st == PGB_OK) st = dalloc(c, &tab->d_T2, T.size());
    if (st != PGB_OK) {
        free_herm_table(tab);
        return st;
    }
    tab->n = nw;
    tab->nrep = (int)(reps.size() / 3);
    tab->M = M;
    PGB_CUDA_TRY(c, cudaMemcpyAsync(tab->d_R, reps.data(), 4 * reps.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(tab->d_T, T.data(), 8 * T.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(tab->d_T2, T2.data(), 4 * T2.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the host vectors go out of scope
    return PGB_OK;
}

void free_herm_table(HermTab *t) {
    dfree(&t->d_R);
    dfree(&t->d_T);
    dfree(&t->d_T2);
    t->n = t->nrep = t->M = 0;
}

// Packed Hermitian X(k) [np][n^2] at np points (crystal coordinates).
pgb_status launch_herm_sum(pgb_ctx *c, const HermTab &t, const double *d_pts, int64_t np, double *d_out) {
    if (np == 0) return PGB_OK;
    if (!t.d_T) {
        c->err = "herm_sum: no cos/sin table";
        return PGB_ESTATE;
    }
    const int ncol = t.n * t.n;
    const int M = t.M;
    const size_t smem = M <= kHermMaxM ? (size_t)3 * (2 * M + 1) * HS_P * sizeof(float4) : 0;
    const dim3 grid(div_up(np, HS_P), div_up(ncol, HS_C));
    // static buffers (Ah, Al, Bh, Bl) plus the dynamic tables above 48 KB need the opt-in
    constexpr size_t kStatic = 4 * (size_t)HS_K * HS_P * sizeof(float);
    if (smem + kStatic > 48 * 1024)
        PGB_CUDA_TRY(c, cudaFuncSetAttribute(k_herm_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_herm_sum<<<grid, 256, smem, c->stream>>>(np, d_pts, t.nrep, t.d_R, M, ncol, t.d_T2, d_out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

// Eigenpairs of count packed Hermitian n x n matrices (2 <= n <= 16): eigenvalues
// ascending in FP64, eigenvectors in FP32 (U32) and/or widened to FP64 (U64).
pgb_status launch_heev_mixed(pgb_ctx *c, int64_t count, int n, const double *d_Hp, double *d_eval, float2 *d_U32,
                             double2 *d_U64, bool refine_vectors) {
    if (count == 0) return PGB_OK;
#define PGB_HEEVM_CASE(NN)                                                                                    \
    case NN: {                                                                                                \
        constexpr int mpb = 64 / JShape<NN>::L;                                                               \
        if (refine_vectors)                                                                                   \
            k_heev_mixed<NN, true><<<div_up(count, mpb), 64, 0, c->stream>>>(count, d_Hp, d_eval, d_U32, d_U64); \
        else                                                                                                  \
            k_heev_mixed<NN, false><<<div_up(count, mpb), 64, 0, c->stream>>>(count, d_Hp, d_eval, d_U32, d_U64); \
        break;                                                                                                \
    }
    switch (n) {
        PGB_HEEVM_CASE(2)
        PGB_HEEVM_CASE(3)
        PGB_HEEVM_CASE(4)
        PGB_HEEVM_CASE(5)
        PGB_HEEVM_CASE(6)
        PGB_HEEVM_CASE(7)
        PGB_HEEVM_CASE(8)
        PGB_HEEVM_CASE(9)
        PGB_HEEVM_CASE(10)
        PGB_HEEVM_CASE(11)
        PGB_HEEVM_CASE(12)
        PGB_HEEVM_CASE(13)
        PGB_HEEVM_CASE(14)
        PGB_HEEVM_CASE(15)
        PGB_HEEVM_CASE(16)
        default:
            c->err = "heev_mixed: n must be 2..16";
            return PGB_EINVAL;
    }
#undef PGB_HEEVM_CASE
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb
