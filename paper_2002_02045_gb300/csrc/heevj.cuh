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

template <int N>
__host__ __device__ inline void heevj_one(double2 (&A)[N][N], double2 (&V)[N][N], double (&w)[N]) {
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) V[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < N; ++r) {
            tot += A[r][r].x * A[r][r].x;
            for (int c = r + 1; c < N; ++c) off += 2.0 * cabs2(A[r][c]);
        }
        tot += off;
        if (!(off > 1e-30 * tot)) break;
        for (int p = 0; p < N - 1; ++p) {
            for (int q = p + 1; q < N; ++q) {
                const double2 b = A[p][q];
                const double ab = sqrt(cabs2(b));
                if (ab == 0.0) continue;
                // e^{-i phi} = conj(b) / |b|
                const double2 em = make_double2(b.x / ab, -b.y / ab);
                const double z = (A[q][q].x - A[p][p].x) / (2.0 * ab);
                double t;
                if (fabs(z) > 1e150)
                    t = 0.5 / z;
                else
                    t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(z * z + 1.0));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                // V-columns of the rotation: col p = (c, -s em), col q = (s, c em)
                const double2 vqp = make_double2(-s * em.x, -s * em.y);
                const double2 vqq = make_double2(c * em.x, c * em.y);
                // A <- A V (columns p, q)
                for (int r = 0; r < N; ++r) {
                    const double2 arp = A[r][p], arq = A[r][q];
                    double2 np_ = make_double2(c * arp.x, c * arp.y);
                    cfma(np_, arq, vqp);
                    double2 nq_ = make_double2(s * arp.x, s * arp.y);
                    cfma(nq_, arq, vqq);
                    A[r][p] = np_;
                    A[r][q] = nq_;
                }
                // A <- V^dagger A (rows p, q)
                for (int r = 0; r < N; ++r) {
                    const double2 apr = A[p][r], aqr = A[q][r];
                    double2 np_ = make_double2(c * apr.x, c * apr.y);
                    cfma_conj(np_, vqp, aqr);
                    double2 nq_ = make_double2(s * apr.x, s * apr.y);
                    cfma_conj(nq_, vqq, aqr);
                    A[p][r] = np_;
                    A[q][r] = nq_;
                }
                A[p][q] = make_double2(0.0, 0.0);
                A[q][p] = make_double2(0.0, 0.0);
                A[p][p].y = 0.0;
                A[q][q].y = 0.0;
                // V <- V Vrot
                for (int r = 0; r < N; ++r) {
                    const double2 vrp = V[r][p], vrq = V[r][q];
                    double2 np_ = make_double2(c * vrp.x, c * vrp.y);
                    cfma(np_, vrq, vqp);
                    double2 nq_ = make_double2(s * vrp.x, s * vrp.y);
                    cfma(nq_, vrq, vqq);
                    V[r][p] = np_;
                    V[r][q] = nq_;
                }
            }
        }
    }
    int order[N];
    for (int i = 0; i < N; ++i) {
        order[i] = i;
        w[i] = A[i][i].x;
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
    double ws[N];
    for (int i = 0; i < N; ++i) ws[i] = w[order[i]];
    for (int i = 0; i < N; ++i) w[i] = ws[i];
    for (int r = 0; r < N; ++r) {
        double2 row[N];
        for (int i = 0; i < N; ++i) row[i] = V[r][order[i]];
        for (int i = 0; i < N; ++i) V[r][i] = row[i];
    }
}

}  // namespace pgb
