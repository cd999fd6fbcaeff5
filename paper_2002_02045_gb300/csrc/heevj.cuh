// Cyclic Jacobi eigensolver for small complex Hermitian matrices, FP64.
//
// Diagonalises H^(W)(k) (Sec. 2.2.1, Eq. wannier_3) and the mass-scaled
// dynamical matrix D(q) (Sec. 2.2.2, Eq. IFC2).  Each rotation first removes
// the phase of the pivot element A_pq = |b| e^{i phi} with diag(1, e^{-i phi})
// on (p, q), then applies the real Jacobi rotation that zeroes the now real
// pivot: V = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on columns (p, q), with
// t = tan(theta) = sgn(z) / (|z| + sqrt(z^2 + 1)), z = (A_qq - A_pp) / (2|b|).
// Sweeps run until the off-diagonal mass is below 1e-30 of the total (at most
// kMaxSweeps sweeps).  Eigenvalues are returned ascending (ties keep their
// original order) and V's columns are the matching eigenvectors, so that
// A = V diag(w) V^dagger.
#pragma once
#include "cplx.cuh"

namespace pgb {

constexpr int kMaxSweeps = 40;

// Matrix entries are held as separate real / imaginary arrays, row-major,
// with the sweep loops kept rolled so that the working set stays small.
template <int N>
__host__ __device__ inline void heevj_one(double (&ar)[N * N], double (&ai)[N * N], double (&vr)[N * N],
                                          double (&vi)[N * N], double (&w)[N]) {
    for (int r = 0; r < N * N; ++r) {
        vr[r] = 0.0;
        vi[r] = 0.0;
    }
    for (int r = 0; r < N; ++r) vr[r * N + r] = 1.0;
#pragma unroll 1
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < N; ++r) {
            tot += ar[r * N + r] * ar[r * N + r];
            for (int c = r + 1; c < N; ++c) off += 2.0 * (ar[r * N + c] * ar[r * N + c] + ai[r * N + c] * ai[r * N + c]);
        }
        tot += off;
        if (!(off > 1e-30 * tot)) break;
#pragma unroll 1
        for (int p = 0; p < N - 1; ++p) {
#pragma unroll 1
            for (int q = p + 1; q < N; ++q) {
                const double br = ar[p * N + q], bi = ai[p * N + q];
                const double ab = sqrt(br * br + bi * bi);
                if (ab == 0.0) continue;
                // e^{-i phi} = conj(b) / |b|
                const double er = br / ab, ei = -bi / ab;
                const double z = (ar[q * N + q] - ar[p * N + p]) / (2.0 * ab);
                double t;
                if (fabs(z) > 1e150)
                    t = 0.5 / z;
                else
                    t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(z * z + 1.0));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                // rotation columns: col p = (c, -s e), col q = (s, c e), e = e^{-i phi}
                const double vqp_r = -s * er, vqp_i = -s * ei;
                const double vqq_r = c * er, vqq_i = c * ei;
                // A <- A V (columns p, q)
                for (int r = 0; r < N; ++r) {
                    const double xr = ar[r * N + p], xi = ai[r * N + p];
                    const double yr = ar[r * N + q], yi = ai[r * N + q];
                    ar[r * N + p] = c * xr + (yr * vqp_r - yi * vqp_i);
                    ai[r * N + p] = c * xi + (yr * vqp_i + yi * vqp_r);
                    ar[r * N + q] = s * xr + (yr * vqq_r - yi * vqq_i);
                    ai[r * N + q] = s * xi + (yr * vqq_i + yi * vqq_r);
                }
                // A <- V^dagger A (rows p, q): conj(vqp), conj(vqq) multiply row q
                for (int r = 0; r < N; ++r) {
                    const double xr = ar[p * N + r], xi = ai[p * N + r];
                    const double yr = ar[q * N + r], yi = ai[q * N + r];
                    ar[p * N + r] = c * xr + (vqp_r * yr + vqp_i * yi);
                    ai[p * N + r] = c * xi + (vqp_r * yi - vqp_i * yr);
                    ar[q * N + r] = s * xr + (vqq_r * yr + vqq_i * yi);
                    ai[q * N + r] = s * xi + (vqq_r * yi - vqq_i * yr);
                }
                ar[p * N + q] = 0.0;
                ai[p * N + q] = 0.0;
                ar[q * N + p] = 0.0;
                ai[q * N + p] = 0.0;
                ai[p * N + p] = 0.0;
                ai[q * N + q] = 0.0;
                // V <- V Vrot
                for (int r = 0; r < N; ++r) {
                    const double xr = vr[r * N + p], xi = vi[r * N + p];
                    const double yr = vr[r * N + q], yi = vi[r * N + q];
                    vr[r * N + p] = c * xr + (yr * vqp_r - yi * vqp_i);
                    vi[r * N + p] = c * xi + (yr * vqp_i + yi * vqp_r);
                    vr[r * N + q] = s * xr + (yr * vqq_r - yi * vqq_i);
                    vi[r * N + q] = s * xi + (yr * vqq_i + yi * vqq_r);
                }
            }
        }
    }
    int order[N];
    for (int i = 0; i < N; ++i) {
        order[i] = i;
        w[i] = ar[i * N + i];
    }
    // stable insertion sort, ascending
    for (int i = 1; i < N; ++i) {
        const int oi = order[i];
        const double wi = w[oi];
        int j = i - 1;
        while (j >= 0 && w[order[j]] > wi) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = oi;
    }
    // permute: eigenvalues into w, eigenvector columns into (ar, ai) as scratch, then back
    for (int i = 0; i < N; ++i) ar[i] = w[order[i]];
    for (int i = 0; i < N; ++i) w[i] = ar[i];
    for (int r = 0; r < N; ++r)
        for (int i = 0; i < N; ++i) {
            ar[r * N + i] = vr[r * N + order[i]];
            ai[r * N + i] = vi[r * N + order[i]];
        }
    for (int r = 0; r < N * N; ++r) {
        vr[r] = ar[r];
        vi[r] = ai[r];
    }
}

}  // namespace pgb
