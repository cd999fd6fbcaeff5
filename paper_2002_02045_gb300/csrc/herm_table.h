// Cos/sin coefficient table of a Hermitian Fourier sum (host code, no CUDA).
//
// Sec. 2.2.1, Eq. wannier_3 (H(k) = sum_R e^{ik.R} H(R)) and Sec. 2.2.2, Eq. IFC2
// (the mass-scaled D(q)).  The Hermitian part of X(k) = sum_R e^{ik.R} X(R) is,
// for a set of R closed under inversion,
//   X(k) = sum_{R in S} cos(k.R) C_R + sin(k.R) S_R,
//   C_R = A(R) + A(-R),  S_R = B(R) - B(-R)   (C_0 = A(0), S_0 = 0),
//   A(Y) = (X(Y) + X(Y)^dagger) / 2,  B(Y) = i (X(Y) - X(Y)^dagger) / 2,
// with S = {0} and every R that is lexicographically positive.  C_R and S_R are
// Hermitian; a row of the table holds their upper triangle packed as n real
// diagonal entries, then (re, im) of (i, j), i < j, row by row (n^2 reals).
#pragma once
#include <cstdint>
#include <cstdlib>
#include <map>
#include <tuple>
#include <vector>

namespace pgb {

// Packed column of entry (i, j), i < j, of an n x n Hermitian matrix (its real part;
// the imaginary part follows).
inline int herm_packed_col(int n, int i, int j) { return n + 2 * (i * n - (i * (i + 1)) / 2 + (j - i - 1)); }

// X: [nR][n][n] complex, interleaved (re, im).  Fills reps [nrep][3], T [2 nrep][n*n]
// (row 2r: C_R, row 2r+1: S_R) and M = max |R_d| over the representatives.
// Returns false (outputs unspecified) when the R list is not closed under inversion.
inline bool herm_table_host(const int32_t *R, const double *X, int nR, int n, std::vector<int32_t> &reps,
                            std::vector<double> &T, int &M) {
    using Key = std::tuple<int, int, int>;
    std::map<Key, int> idx;
    for (int r = 0; r < nR; ++r) idx[Key(R[3 * r], R[3 * r + 1], R[3 * r + 2])] = r;
    const int ncol = n * n;
    reps.clear();
    T.clear();
    M = 0;
    // A(Y)_ij and B(Y)_ij from X(Y)_ij and conj(X(Y)_ji)
    auto parts = [&](int Y, int i, int j, double A[2], double B[2]) {
        const double hr = X[2 * ((size_t)Y * ncol + i * n + j)], hi = X[2 * ((size_t)Y * ncol + i * n + j) + 1];
        const double tr = X[2 * ((size_t)Y * ncol + j * n + i)], ti = X[2 * ((size_t)Y * ncol + j * n + i) + 1];
        A[0] = 0.5 * (hr + tr);
        A[1] = 0.5 * (hi - ti);
        const double dr = hr - tr, di = hi + ti;   // X_ij - conj(X_ji)
        B[0] = -0.5 * di;                          // i * d / 2
        B[1] = 0.5 * dr;
    };
    for (int r = 0; r < nR; ++r) {
        const int x = R[3 * r], y = R[3 * r + 1], z = R[3 * r + 2];
        const bool zero = x == 0 && y == 0 && z == 0;
        const bool pos = x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0)));
        if (!zero && !pos) continue;
        int rn = r;
        if (!zero) {
            auto it = idx.find(Key(-x, -y, -z));
            if (it == idx.end()) return false;
            rn = it->second;
        }
        reps.push_back(x);
        reps.push_back(y);
        reps.push_back(z);
        const int ax = std::abs(x), ay = std::abs(y), az = std::abs(z);
        if (ax > M) M = ax;
        if (ay > M) M = ay;
        if (az > M) M = az;
        std::vector<double> Cr(ncol, 0.0), Sr(ncol, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                double Ap[2], Bp[2], C[2], Sv[2];
                parts(r, i, j, Ap, Bp);
                if (zero) {
                    C[0] = Ap[0];
                    C[1] = Ap[1];
                    Sv[0] = Sv[1] = 0.0;
                } else {
                    double An[2], Bn[2];
                    parts(rn, i, j, An, Bn);
                    C[0] = Ap[0] + An[0];
                    C[1] = Ap[1] + An[1];
                    Sv[0] = Bp[0] - Bn[0];
                    Sv[1] = Bp[1] - Bn[1];
                }
                if (i == j) {
                    Cr[i] = C[0];
                    Sr[i] = Sv[0];
                } else {
                    const int p = herm_packed_col(n, i, j);
                    Cr[p] = C[0];
                    Cr[p + 1] = C[1];
                    Sr[p] = Sv[0];
                    Sr[p + 1] = Sv[1];
                }
            }
        T.insert(T.end(), Cr.begin(), Cr.end());
        T.insert(T.end(), Sr.begin(), Sr.end());
    }
    return true;
}

}  // namespace pgb
