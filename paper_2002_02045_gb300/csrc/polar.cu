// Long-range (Froehlich) e-ph coupling of polar materials (Sec. 2.2.4, Eqs.
// e_ph_long and smooth_phase).
//
// In the Wannier gauge, with the smooth-phase bra-ket, the long-range part of
// g~^{ka}_ij(k, q) is L^{ka}(q) delta_ij, where
//   L^{ka}(q) = i (e^2 / (eps_0 Omega)) sum_{G, q+G != 0} [(q+G).Z*_k]_a
//               e^{-i tau_k.(q+G)} e^{-(q+G).eps.(q+G) / (4 Lambda)} / ((q+G).eps.(q+G)),
// summed over every G whose exponent (q+G).eps.(q+G)/(4 Lambda) is at most
// kEwaldCut.  After U(k) is folded in, the term adds L^{ka}(q) U_in(k) to the
// R_p sum C[q][n][ka][i]; the library therefore appends nmode rows to that
// sum: row nRgp + k'a' of the q table holds L^{k'a'}(q), and the same row of
// the folded g holds delta(ka, k'a') U_in(k).  Every path that forms the R_p
// sum (tensor-core, SIMT, arbitrary points, the list builder) then includes
// the long-range term with no other change.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

struct EwaldArgs {
    int64_t npts;
    const int32_t *idx;      // grid point indices (null: all points of the grid) ...
    int grid[3];
    const double *pts;       // ... or explicit crystal coordinates [npts][3]
    double B[9];             // reciprocal vectors (rows), 1/bohr
    double eps[9];
    double inv4lam, cut4lam; // 1 / (4 Lambda), 4 Lambda kEwaldCut
    double pref;             // e^2 / (eps_0 Omega), eV / bohr^2
    int nat;
    const double *tau;       // [nat][3] bohr
    const double *zstar;     // [nat][3 beta][3 alpha]
    int nG;
    const int32_t *gvec;     // [nG][3] integer candidates
    void *out;               // double2 or float2, row p at p * ld + col0
    int64_t ld;
    int col0;
    int fp32;
};

// One warp per point.  The candidates G are screened 32 at a time in FP32 (the
// exponent with a relative margin of 1e-4, far above the FP32 error of ~1e-6), the
// survivors (~60 of 1331 candidates for the zincblende polar model, 8 bands, a = 10.68
// bohr) are compacted into a per-warp
// list by ballot, and the list is evaluated 32 terms at a time in FP64 (every
// lane busy), so the FP64 work is that of the surviving terms only.  Each lane
// sums its terms; the lanes' sums are then added by a butterfly.
constexpr int kEwWarps = 8;
__global__ void __launch_bounds__(32 * kEwWarps) k_ewald(EwaldArgs p) {
    __shared__ int list_s[kEwWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *list = list_s[wid];
    const int64_t t = (int64_t)blockIdx.x * kEwWarps + wid;
    if (t >= p.npts) return;   // warp-uniform
    double q[3];
    if (p.pts) {
        q[0] = p.pts[3 * t];
        q[1] = p.pts[3 * t + 1];
        q[2] = p.pts[3 * t + 2];
    } else {
        const int64_t id = p.idx ? (int64_t)p.idx[t] : t;
        const int i3 = (int)(id % p.grid[2]), i2 = (int)((id / p.grid[2]) % p.grid[1]);
        const int i1 = (int)(id / ((int64_t)p.grid[1] * p.grid[2]));
        q[0] = (double)i1 / p.grid[0];
        q[1] = (double)i2 / p.grid[1];
        q[2] = (double)i3 / p.grid[2];
    }
    const int nm = 3 * p.nat;
    double ar[kMaxNmode], ai[kMaxNmode];
#pragma unroll
    for (int j = 0; j < kMaxNmode; ++j) {
        ar[j] = 0.0;
        ai[j] = 0.0;
    }
    float Bf[9], Ef[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Bf[i] = (float)p.B[i];
        Ef[i] = (float)p.eps[i];
    }
    const float cutf = (float)(p.cut4lam * (1.0 + 1e-4));
    // one surviving term, exactly as the FP64 definition
    auto term = [&](int g) {
        const double m0 = q[0] + p.gvec[3 * g], m1 = q[1] + p.gvec[3 * g + 1], m2 = q[2] + p.gvec[3 * g + 2];
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = m0 * p.B[a] + m1 * p.B[3 + a] + m2 * p.B[6 + a];
        double x = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) x += v[a] * p.eps[3 * a + b] * v[b];
        if (!(x > 0.0) || x > p.cut4lam) return;
        const double w = exp(-x * p.inv4lam) / x;
#pragma unroll
        for (int k = 0; k < kMaxNmode / 3; ++k) {
            if (k >= p.nat) break;
            const double th = v[0] * p.tau[3 * k] + v[1] * p.tau[3 * k + 1] + v[2] * p.tau[3 * k + 2];
            double s, c;
            sincos(th, &s, &c);
            const double wr = w * c, wi = -w * s;       // w e^{-i th}
            const double *Z = p.zstar + 9 * k;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double vz = v[0] * Z[a] + v[1] * Z[3 + a] + v[2] * Z[6 + a];
                ar[3 * k + a] += wr * vz;
                ai[3 * k + a] += wi * vz;
            }
        }
    };
    const float q0 = (float)q[0], q1 = (float)q[1], q2 = (float)q[2];
    int cnt = 0;   // warp-uniform length of the survivor list
    for (int g0 = 0; g0 < p.nG; g0 += 32) {
        const int g = g0 + lane;
        bool keep = false;
        if (g < p.nG) {
            const float m0 = q0 + (float)p.gvec[3 * g], m1 = q1 + (float)p.gvec[3 * g + 1],
                        m2 = q2 + (float)p.gvec[3 * g + 2];
            float v[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = m0 * Bf[a] + m1 * Bf[3 + a] + m2 * Bf[6 + a];
            float x = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) x += v[a] * Ef[3 * a + b] * v[b];
            keep = x <= cutf;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) list[cnt + __popc(bal & ((1u << lane) - 1u))] = g;
        cnt += __popc(bal);
        __syncwarp();
        if (cnt >= 32) {
            term(list[cnt - 32 + lane]);
            cnt -= 32;
        }
        __syncwarp();
    }
    if (lane < cnt) term(list[lane]);
    // warp sums, then i * pref
#pragma unroll
    for (int j = 0; j < kMaxNmode; ++j) {
        if (j >= nm) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar[j] += __shfl_xor_sync(0xffffffffu, ar[j], o);
            ai[j] += __shfl_xor_sync(0xffffffffu, ai[j], o);
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxNmode; ++j) {
        if (j >= nm) break;
        if (lane != j) continue;
        const double re = -p.pref * ai[j], im = p.pref * ar[j];
        if (p.fp32)
            reinterpret_cast<float2 *>(p.out)[t * p.ld + p.col0 + j] = make_float2((float)re, (float)im);
        else
            reinterpret_cast<double2 *>(p.out)[t * p.ld + p.col0 + j] = make_double2(re, im);
    }
}

template <typename T2>
__global__ void k_copy_cols(int64_t npts, const int32_t *__restrict__ idx, int ncols, const double2 *__restrict__ src,
                            T2 *__restrict__ out, int64_t ld, int col0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts * ncols) return;
    const int64_t p = t / ncols;
    const int j = (int)(t % ncols);
    const double2 v = src[(idx ? (int64_t)idx[p] : p) * ncols + j];
    T2 o;
    o.x = v.x;
    o.y = v.y;
    out[p * ld + col0 + j] = o;
}

EwaldArgs ewald_args(const pgb_ctx *c) {
    EwaldArgs a;
    a.npts = 0;
    a.idx = nullptr;
    a.grid[0] = a.grid[1] = a.grid[2] = 1;
    a.pts = nullptr;
    for (int i = 0; i < 9; ++i) {
        a.B[i] = c->rec[i];
        a.eps[i] = c->eps_inf[i];
    }
    a.inv4lam = 1.0 / (4.0 * c->ewald_lambda);
    a.cut4lam = 4.0 * c->ewald_lambda * kEwaldCut;
    a.pref = 4.0 * kPi * kHartreeEv / c->omega;
    a.nat = c->nat;
    a.tau = c->d_polar;
    a.zstar = c->d_polar + 3 * c->nat;
    a.nG = c->nG;
    a.gvec = c->d_gvec;
    a.out = nullptr;
    a.ld = c->nm;
    a.col0 = 0;
    a.fp32 = 0;
    return a;
}

}  // namespace

pgb_status launch_ewald_pts(pgb_ctx *c, const double *d_pts, int64_t npts, void *out, int64_t ld, int col0,
                            bool fp32) {
    if (npts == 0) return PGB_OK;
    EwaldArgs a = ewald_args(c);
    a.npts = npts;
    a.pts = d_pts;
    a.out = out;
    a.ld = ld;
    a.col0 = col0;
    a.fp32 = fp32 ? 1 : 0;
    k_ewald<<<div_up(npts, kEwWarps), 32 * kEwWarps, 0, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status polar_grid_table(pgb_ctx *c) {
    dfree(&c->d_polarL);
    if (!c->polar || !c->has_grids) return PGB_OK;
    pgb_status st;
    if ((st = dalloc(c, &c->d_polarL, (size_t)c->Nq * c->nm)) != PGB_OK) return st;
    EwaldArgs a = ewald_args(c);
    a.npts = c->Nq;
    for (int d = 0; d < 3; ++d) a.grid[d] = c->qg[d];
    a.out = c->d_polarL;
    a.ld = c->nm;
    k_ewald<<<div_up(c->Nq, kEwWarps), 32 * kEwWarps, 0, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_qtable_grid(pgb_ctx *c, const int32_t *d_idx, int64_t npts, void *out, bool fp32) {
    pgb_status st;
    if ((st = launch_phase_grid(c, c->qg, d_idx, npts, c->d_Rgp, c->nRgp, out, fp32, c->nKp)) != PGB_OK) return st;
    if (!c->polar || npts == 0) return PGB_OK;
    const int64_t n = npts * c->nm;
    if (fp32)
        k_copy_cols<float2><<<div_up(n, 256), 256, 0, c->stream>>>(npts, d_idx, c->nm, c->d_polarL, (float2 *)out,
                                                                    c->nKp, c->nRgp);
    else
        k_copy_cols<double2><<<div_up(n, 256), 256, 0, c->stream>>>(npts, d_idx, c->nm, c->d_polarL,
                                                                     (double2 *)out, c->nKp, c->nRgp);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_qtable_pts(pgb_ctx *c, const double *d_pts, int64_t npts, void *out, bool fp32) {
    pgb_status st;
    if ((st = launch_phase_pts(c, d_pts, npts, c->d_Rgp, c->nRgp, out, fp32, c->nKp)) != PGB_OK) return st;
    if (!c->polar) return PGB_OK;
    return launch_ewald_pts(c, d_pts, npts, out, c->nKp, c->nRgp, fp32);
}

// Integer G candidates covering every q + G with (q+G).eps.(q+G) <= 4 Lambda kEwaldCut
// for q anywhere in [-1, 1]^3 (crystal coordinates).
std::vector<int32_t> ewald_candidates(const double lat[9], const double eps[9], double lambda) {
    // smallest eigenvalue of eps (symmetric 3x3) by a few Jacobi rotations on the host
    double a[9];
    for (int i = 0; i < 9; ++i) a[i] = 0.5 * (eps[i] + eps[3 * (i % 3) + i / 3]);
    for (int sweep = 0; sweep < 50; ++sweep)
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = a[3 * p + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double th = 0.5 * std::atan2(2 * apq, a[3 * q + q] - a[3 * p + p]);
                const double cs = std::cos(th), sn = std::sin(th);
                for (int k = 0; k < 3; ++k) {   // columns p, q
                    const double x = a[3 * k + p], y = a[3 * k + q];
                    a[3 * k + p] = cs * x - sn * y;
                    a[3 * k + q] = sn * x + cs * y;
                }
                for (int k = 0; k < 3; ++k) {   // rows p, q
                    const double x = a[3 * p + k], y = a[3 * q + k];
                    a[3 * p + k] = cs * x - sn * y;
                    a[3 * q + k] = sn * x + cs * y;
                }
            }
    const double emin = std::min(a[0], std::min(a[4], a[8]));
    const double vmax = std::sqrt(4.0 * lambda * kEwaldCut / emin);
    double amax = 0.0;
    for (int i = 0; i < 3; ++i)
        amax = std::max(amax, std::sqrt(lat[3 * i] * lat[3 * i] + lat[3 * i + 1] * lat[3 * i + 1] +
                                        lat[3 * i + 2] * lat[3 * i + 2]));
    const int nmax = (int)std::ceil(vmax * amax / (2 * kPi)) + 2;
    std::vector<int32_t> g;
    for (int i = -nmax; i <= nmax; ++i)
        for (int j = -nmax; j <= nmax; ++j)
            for (int k = -nmax; k <= nmax; ++k) {
                g.push_back(i);
                g.push_back(j);
                g.push_back(k);
            }
    return g;
}

}  // namespace pgb
