// Band velocities (Sec. 2.2.1, Eqs. velocity and wannier_4), the iterative
// solution of the linearised BTE (Sec. 2.1.2, Eqs. BTE_lin, BTE_iter, BTE_W)
// and the mobility (Eq. cond).
//
// Velocities: H_a(k) = sum_R e^{ik.R} [i R^a H(R)] is one FP64 complex GEMM of
// the k phase table with the table i R^a H(R) built by set_lattice (R^a
// Cartesian); a thread per (k, a) forms [U^dagger H_a U]_nn and, for bands
// degenerate within kDegTol, the eigenvalues of the restricted block.
//
// BTE: the list of pgb_build_collision_grid (window states, rows sorted) gives
// W per entry; F^{i+1}_s = tau_s v_s + tau_s sum_{e in row s} W_e F^i_{col e} is a
// CSR product per iteration, one 256-thread block per non-empty row.  The
// iteration matrix tau W of a window that keeps most of its scattering inside
// has a spectral radius within 1e-2 .. 1e-5 of one, so F amplifies any error
// of W by 1e2 .. 1e5: W, F and the products are FP64 here (the FP64 rate is
// enough for one product per entry per iteration).  The largest change of
// any component is reduced with an integer atomic max on the bits of a
// non-negative double (order independent).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "coeffs.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }
constexpr double kDegTol = 1e-6;   // eV
constexpr double kBohrM = 0.529177210903e-10;

__global__ void k_make_hd(int nRH, int nw, const int32_t *__restrict__ R, double l0, double l1, double l2, double l3,
                          double l4, double l5, double l6, double l7, double l8, const double2 *__restrict__ H,
                          double2 *__restrict__ Hd) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw2 = (int64_t)nw * nw;
    if (t >= (int64_t)nRH * 3 * nw2) return;
    const int64_t r = t / (3 * nw2);
    const int a = (int)((t / nw2) % 3);
    const int64_t ij = t % nw2;
    const double L[9] = {l0, l1, l2, l3, l4, l5, l6, l7, l8};
    const double Ra = R[3 * r] * L[a] + R[3 * r + 1] * L[3 + a] + R[3 * r + 2] * L[6 + a];   // Cartesian bohr
    const double2 h = H[r * nw2 + ij];
    Hd[t] = make_double2(-Ra * h.y, Ra * h.x);   // i R^a H
}

// Eigenvalues (ascending) of a small Hermitian matrix by cyclic complex Jacobi:
// each pivot's phase is removed by diag(1, e^{-i phi}), then a real rotation
// zeroes it.
__device__ void herm_eigvals(int d, double *ar, double *ai, double *w) {
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < d; ++r) {
            tot += ar[r * d + r] * ar[r * d + r];
            for (int c = r + 1; c < d; ++c) off += 2.0 * (ar[r * d + c] * ar[r * d + c] + ai[r * d + c] * ai[r * d + c]);
        }
        tot += off;
        if (!(off > 1e-30 * tot)) break;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                const double br = ar[p * d + q], bi = ai[p * d + q];
                const double ab = hypot(br, bi);
                if (ab == 0.0) continue;
                const double cr = br / ab, ci = bi / ab;     // e^{i phi}
                for (int j = 0; j < d; ++j) {                // row q times e^{i phi}
                    const double xr = ar[q * d + j], xi = ai[q * d + j];
                    ar[q * d + j] = xr * cr - xi * ci;
                    ai[q * d + j] = xr * ci + xi * cr;
                }
                for (int i = 0; i < d; ++i) {                // column q times e^{-i phi}
                    const double xr = ar[i * d + q], xi = ai[i * d + q];
                    ar[i * d + q] = xr * cr + xi * ci;
                    ai[i * d + q] = xi * cr - xr * ci;
                }
                const double app = ar[p * d + p], aqq = ar[q * d + q], b = ar[p * d + q];
                const double z = (aqq - app) / (2.0 * b);
                const double t = (z >= 0 ? 1.0 : -1.0) / (fabs(z) + sqrt(z * z + 1.0));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int i = 0; i < d; ++i) {                // columns p, q
                    const double xr = ar[i * d + p], xi = ai[i * d + p], yr = ar[i * d + q], yi = ai[i * d + q];
                    ar[i * d + p] = c * xr - s * yr;
                    ai[i * d + p] = c * xi - s * yi;
                    ar[i * d + q] = s * xr + c * yr;
                    ai[i * d + q] = s * xi + c * yi;
                }
                for (int j = 0; j < d; ++j) {                // rows p, q
                    const double xr = ar[p * d + j], xi = ai[p * d + j], yr = ar[q * d + j], yi = ai[q * d + j];
                    ar[p * d + j] = c * xr - s * yr;
                    ai[p * d + j] = c * xi - s * yi;
                    ar[q * d + j] = s * xr + c * yr;
                    ai[q * d + j] = s * xi + c * yi;
                }
            }
    }
    for (int i = 0; i < d; ++i) w[i] = ar[i * d + i];
    for (int i = 1; i < d; ++i)   // insertion sort
        for (int j = i; j > 0 && w[j] < w[j - 1]; --j) {
            const double x = w[j];
            w[j] = w[j - 1];
            w[j - 1] = x;
        }
}

// thread per (k, a): v[k][n][a] in m/s
__global__ void k_velocity(int64_t nk, const int32_t *__restrict__ kidx, int nw, const double2 *__restrict__ Hk,
                           const double2 *__restrict__ U, const double *__restrict__ eps, double *__restrict__ v) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk * 3) return;
    const int64_t kb = t / 3;
    const int a = (int)(t % 3);
    const int64_t k = kidx[kb];
    const int64_t nw2 = (int64_t)nw * nw;
    const double2 *H = Hk + (kb * 3 + a) * nw2;
    const double2 *u = U + k * nw2;          // u[i * nw + n] = U_in
    const double *e = eps + k * nw;
    const double conv = kBohrM / kHbarEvS;    // eV bohr / hbar -> m/s
    double hu_r[kMaxNw], hu_i[kMaxNw];
    int n = 0;
    while (n < nw) {
        int end = n + 1;
        while (end < nw && e[end] - e[end - 1] <= kDegTol) ++end;
        const int d = end - n;
        double ar[kMaxNw * kMaxNw], ai[kMaxNw * kMaxNw];
        for (int cn = 0; cn < d; ++cn) {
            const int col = n + cn;
            for (int i = 0; i < nw; ++i) {       // (H U)_i,col
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < nw; ++j) {
                    const double2 h = H[i * nw + j], x = u[j * nw + col];
                    sr += h.x * x.x - h.y * x.y;
                    si += h.x * x.y + h.y * x.x;
                }
                hu_r[i] = sr;
                hu_i[i] = si;
            }
            for (int rn = 0; rn < d; ++rn) {     // (U^dagger H U)_row,col
                const int row = n + rn;
                double sr = 0.0, si = 0.0;
                for (int i = 0; i < nw; ++i) {
                    const double2 x = u[i * nw + row];
                    sr += x.x * hu_r[i] + x.y * hu_i[i];
                    si += x.x * hu_i[i] - x.y * hu_r[i];
                }
                ar[rn * d + cn] = sr;
                ai[rn * d + cn] = si;
            }
        }
        if (d == 1) {
            v[(kb * nw + n) * 3 + a] = ar[0] * conv;
        } else {
            for (int r = 0; r < d; ++r)          // exact Hermitian symmetry of the block
                for (int c2 = r + 1; c2 < d; ++c2) {
                    const double mr = 0.5 * (ar[r * d + c2] + ar[c2 * d + r]);
                    const double mi = 0.5 * (ai[r * d + c2] - ai[c2 * d + r]);
                    ar[r * d + c2] = mr;
                    ai[r * d + c2] = mi;
                    ar[c2 * d + r] = mr;
                    ai[c2 * d + r] = -mi;
                }
            for (int r = 0; r < d; ++r) ai[r * d + r] = 0.0;
            double w[kMaxNw];
            herm_eigvals(d, ar, ai, w);
            for (int r = 0; r < d; ++r) v[(kb * nw + n + r) * 3 + a] = w[r] * conv;
        }
        n = end;
    }
}

// W_e / N_q per entry (Eq. BTE_W), FP64 arithmetic, stored FP32
struct WArgs {
    int64_t nnz;
    const int32_t *row, *col, *mode;
    const float *g2;
    CoeffGeom g;
    const double *eps_state;
    double mu;
    double *w;
};

__global__ void k_bte_weights(WArgs p) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.nnz) return;
    double de, da, N;
    double w = 0.0;
    if (coll_factors(p.g, p.row[e], p.col[e], p.mode[e], de, da, N)) {
        const double f = 1.0 / (exp((p.eps_state[p.col[e]] - p.mu) / (kBoltzEvK * p.g.T)) + 1.0);
        w = p.g.scale * (double)p.g2[e] * (de * (1.0 + N - f) + da * (N + f));
    }
    p.w[e] = w;
}

// per state: tau, F^0 = tau v (window states with Gamma > 0), FP32 copies
__global__ void k_bte_init(int64_t ns, int nbnd, int band_lo, int nw, const uint8_t *__restrict__ inwin,
                           const int32_t *__restrict__ kpos, const double *__restrict__ gamma,
                           const double *__restrict__ vel, double *__restrict__ tau, double *__restrict__ v,
                           double *__restrict__ F0, double *__restrict__ F) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int64_t k = s / nbnd;
    const int n = (int)(s % nbnd) + band_lo;
    double t = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    const int32_t kp = kpos[k];
    if (inwin[s] && kp >= 0) {
        const double g = gamma[(int64_t)kp * nw + n];
        t = g > 0.0 ? 1.0 / g : 0.0;
        const double *vv = vel + ((int64_t)kp * nw + n) * 3;
        vx = vv[0];
        vy = vv[1];
        vz = vv[2];
    }
    tau[s] = t;
    v[3 * s] = vx;
    v[3 * s + 1] = vy;
    v[3 * s + 2] = vz;
    const double f0x = t * vx, f0y = t * vy, f0z = t * vz;
    F0[3 * s] = f0x;
    F0[3 * s + 1] = f0y;
    F0[3 * s + 2] = f0z;
    F[3 * s] = f0x;
    F[3 * s + 1] = f0y;
    F[3 * s + 2] = f0z;
}

struct IterArgs {
    int64_t nrows;
    const int32_t *rows;
    const int64_t *rowptr;
    const int32_t *col;
    const double *w;
    const double *tau;
    const double *F0;
    const double *Fold;
    double *Fnew;
    unsigned long long *maxdiff;   // bits of a non-negative double
};

constexpr int kIterThreads = 256;

__global__ void __launch_bounds__(kIterThreads) k_bte_iter(IterArgs p) {
    __shared__ double red[3][kIterThreads / 32];
    const int64_t r = blockIdx.x;
    if (r >= p.nrows) return;
    const int s = p.rows[r];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t beg = p.rowptr[s], end = p.rowptr[s + 1];
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t e = beg + t; e < end; e += kIterThreads) {
        const double w = p.w[e];
        const double *f = p.Fold + 3 * (int64_t)p.col[e];
        v[0] = fma(w, __ldg(f), v[0]);
        v[1] = fma(w, __ldg(f + 1), v[1]);
        v[2] = fma(w, __ldg(f + 2), v[2]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
        if (lane == 0) red[i][warp] = v[i];
    }
    __syncthreads();
    if (t == 0) {
        double S[3] = {0, 0, 0};
        for (int w = 0; w < kIterThreads / 32; ++w)
            for (int i = 0; i < 3; ++i) S[i] += red[i][w];
        const double ts = p.tau[s];
        double diff = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double fn = p.F0[3 * s + i] + ts * S[i];
            diff = fmax(diff, fabs(fn - p.Fold[3 * s + i]));
            p.Fnew[3 * s + i] = fn;
        }
        atomicMax(p.maxdiff, (unsigned long long)__double_as_longlong(diff));
    }
}

// per block: sum over its states of w v^a F^b (9) and f (1), w = f (1 - f) / kT
constexpr int kMobThreads = 256;
__global__ void k_mobility(int64_t ns, const uint8_t *__restrict__ inwin, const double *__restrict__ eps_state,
                           double mu, double T, const double *__restrict__ v, const double *__restrict__ F,
                           double *__restrict__ partial) {
    __shared__ double red[10][kMobThreads / 32];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[10];
    for (int i = 0; i < 10; ++i) acc[i] = 0.0;
    if (s < ns && inwin[s]) {
        const double kT = kBoltzEvK * T;
        const double f = 1.0 / (exp((eps_state[s] - mu) / kT) + 1.0);
        const double w = f * (1.0 - f) / kT;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc[3 * a + b] = w * v[3 * s + a] * F[3 * s + b];
        acc[9] = f;
    }
    for (int i = 0; i < 10; ++i) {
        double x = acc[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[i][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double x = 0.0;
        for (int w = 0; w < kMobThreads / 32; ++w) x += red[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * 10 + threadIdx.x] = x;
    }
}

pgb_status mobility_sum(pgb_ctx *c, const uint8_t *inwin, double mu, const double *v, const double *F, double out[9],
                        double *nsum) {
    const int64_t ns = c->nstates;
    const unsigned nblk = div_up(ns, kMobThreads);
    double *part = nullptr;
    PGB_CUDA_TRY(c, dev_malloc_async((void **)&part, 80 * (size_t)std::max(1u, nblk), c->stream));
    k_mobility<<<nblk, kMobThreads, 0, c->stream>>>(ns, inwin, c->d_eps_state, mu, c->coll_T, v, F, part);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    std::vector<double> h((size_t)nblk * 10);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), part, 8 * h.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFreeAsync(part, c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("transport: mobility sum: ") + cudaGetErrorString(e);
        return PGB_ECUDA;
    }
    double acc[10] = {0};
    for (unsigned b = 0; b < nblk; ++b)   // fixed order: deterministic
        for (int i = 0; i < 10; ++i) acc[i] += h[(size_t)b * 10 + i];
    *nsum = acc[9];
    for (int i = 0; i < 9; ++i) out[i] = acc[9] > 0.0 ? 1e4 * acc[i] / acc[9] : 0.0;   // m^2 -> cm^2
    return PGB_OK;
}

}  // namespace

pgb_status build_velocity_tables(pgb_ctx *c) {
    const int64_t n = (int64_t)c->nRH * 3 * c->nw * c->nw;
    pgb_status st;
    if ((st = dalloc(c, &c->d_Hd, (size_t)n)) != PGB_OK) return st;
    const double *L = c->lat;
    k_make_hd<<<div_up(n, 256), 256, 0, c->stream>>>(c->nRH, c->nw, c->d_RH, L[0], L[1], L[2], L[3], L[4], L[5], L[6],
                                                      L[7], L[8], c->d_H, c->d_Hd);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status band_velocities(pgb_ctx *c, const int32_t *d_kidx, int64_t nk, double *d_v) {
    if (nk == 0) return PGB_OK;
    const int nw = c->nw;
    const int64_t nw2 = (int64_t)nw * nw;
    const int64_t chunk = 16384;
    double2 *ph = nullptr, *Hk = nullptr;
    PGB_CUDA_TRY(c, dev_malloc_async((void **)&ph, 16 * (size_t)std::min(nk, chunk) * c->nRH, c->stream));
    PGB_CUDA_TRY(c, dev_malloc_async((void **)&Hk, 16 * (size_t)std::min(nk, chunk) * 3 * nw2, c->stream));
    pgb_status st = PGB_OK;
    for (int64_t k0 = 0; k0 < nk && st == PGB_OK; k0 += chunk) {
        const int64_t nb = std::min(chunk, nk - k0);
        st = launch_phase_grid(c, c->kg, d_kidx + k0, nb, c->d_RH, c->nRH, ph, false);
        if (st == PGB_OK)
            st = launch_cgemm(c, false, 1, nb, 3 * nw2, c->nRH, ph, c->nRH, 0, c->d_Hd, 3 * nw2, 0, Hk, 3 * nw2, 0);
        if (st == PGB_OK) {
            k_velocity<<<div_up(nb * 3, 128), 128, 0, c->stream>>>(nb, d_kidx + k0, nw, Hk, c->d_U, c->d_eps,
                                                                   d_v + k0 * nw * 3);
            c->launches++;
            if (cudaGetLastError() != cudaSuccess) {
                c->err = "band_velocities: kernel launch failed";
                st = PGB_ECUDA;
            }
        }
    }
    cudaFreeAsync(ph, c->stream);
    cudaFreeAsync(Hk, c->stream);
    return st;
}

pgb_status transport(pgb_ctx *c, double mu, int precision, int max_iter, double tol, double *mob_rta, double *mob,
                     int64_t *iters_out, double *d_F, double *d_tau) {
    const int64_t ns = c->nstates, nnz = c->nnz;
    const int nbnd = c->band_hi - c->band_lo, nw = c->nw;
    // window states (energies of the list's states against its window) and their k-points
    std::vector<double> es((size_t)ns);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(es.data(), c->d_eps_state, 8 * (size_t)ns, cudaMemcpyDeviceToHost, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<uint8_t> win((size_t)ns, 0);
    std::vector<int32_t> kpos((size_t)c->Nk, -1), klist;
    for (int64_t s = 0; s < ns; ++s) {
        if (!(es[s] >= c->coll_elo && es[s] <= c->coll_ehi)) continue;
        win[s] = 1;
        const int64_t k = s / nbnd;
        if (kpos[k] < 0) {
            kpos[k] = (int32_t)klist.size();
            klist.push_back((int32_t)k);
        }
    }
    const int64_t nkw = (int64_t)klist.size();
    struct Buf {
        pgb_ctx *c;
        std::vector<void *> p;
        bool ok = true;
        void *get(size_t bytes) {
            void *x = nullptr;
            if (dev_malloc_async(&x, std::max<size_t>(bytes, 16), c->stream) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                return nullptr;
            }
            p.push_back(x);
            return x;
        }
        ~Buf() {
            for (void *x : p) cudaFreeAsync(x, c->stream);
        }
    } B{c};
    uint8_t *d_win = (uint8_t *)B.get(ns);
    int32_t *d_kpos = (int32_t *)B.get(4 * (size_t)c->Nk);
    int32_t *d_klist = (int32_t *)B.get(4 * (size_t)std::max<int64_t>(nkw, 1));
    double *d_gamma = (double *)B.get(8 * (size_t)std::max<int64_t>(nkw, 1) * nw);
    double *d_vel = (double *)B.get(24 * (size_t)std::max<int64_t>(nkw, 1) * nw);
    double *tau = (double *)B.get(8 * (size_t)ns), *v = (double *)B.get(24 * (size_t)ns);
    double *F0 = (double *)B.get(24 * (size_t)ns);
    double *F[2] = {(double *)B.get(24 * (size_t)ns), (double *)B.get(24 * (size_t)ns)};
    double *w = (double *)B.get(8 * (size_t)nnz);
    unsigned long long *d_max = (unsigned long long *)B.get(8);
    if (!B.ok) {
        c->err = "transport: device allocation failed";
        return PGB_ENOMEM;
    }
    PGB_CUDA_TRY(c, cudaMemcpyAsync(d_win, win.data(), ns, cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaMemcpyAsync(d_kpos, kpos.data(), 4 * (size_t)c->Nk, cudaMemcpyHostToDevice, c->stream));
    if (nkw) PGB_CUDA_TRY(c, cudaMemcpyAsync(d_klist, klist.data(), 4 * (size_t)nkw, cudaMemcpyHostToDevice, c->stream));
    pgb_status st;
    // tau from the full-grid rates, velocities
    if (nkw) {
        if ((st = pgb_scattering_rates(c, d_klist, nkw, c->coll_T, mu, c->coll_sigma, precision, d_gamma, nullptr)) !=
            PGB_OK)
            return st;
        if ((st = band_velocities(c, d_klist, nkw, d_vel)) != PGB_OK) return st;
    }
    k_bte_init<<<div_up(ns, 256), 256, 0, c->stream>>>(ns, nbnd, c->band_lo, nw, d_win, d_kpos, d_gamma, d_vel, tau, v,
                                                       F0, F[0]);
    PGB_LAUNCH_CHECK(c);
    PGB_CUDA_TRY(c, cudaMemcpyAsync(F[1], F[0], 24 * (size_t)ns, cudaMemcpyDeviceToDevice, c->stream));
    double nsum = 0.0;
    if ((st = mobility_sum(c, d_win, mu, v, F0, mob_rta, &nsum)) != PGB_OK) return st;
    // W per entry
    if (nnz) {
        WArgs a;
        a.nnz = nnz;
        a.row = c->d_coo_row;
        a.col = c->d_coo_col;
        a.mode = c->d_coo_mode;
        a.g2 = c->d_coo_g2;
        a.g = coeff_geom(c);
        a.eps_state = c->d_eps_state;
        a.mu = mu;
        a.w = w;
        k_bte_weights<<<div_up(nnz, 256), 256, 0, c->stream>>>(a);
        PGB_LAUNCH_CHECK(c);
    }
    // largest |F^0| component for the stopping rule
    double f0max = 0.0;
    {
        std::vector<double> h(3 * (size_t)ns);
        PGB_CUDA_TRY(c, cudaMemcpyAsync(h.data(), F0, 24 * (size_t)ns, cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (double x : h) f0max = std::max(f0max, std::fabs(x));
    }
    int64_t it = 0;
    int cur = 0;
    while (it < max_iter && c->nrows_active > 0) {
        PGB_CUDA_TRY(c, cudaMemsetAsync(d_max, 0, 8, c->stream));
        IterArgs p;
        p.nrows = c->nrows_active;
        p.rows = c->d_active_rows;
        p.rowptr = c->d_rowptr;
        p.col = c->d_col;
        p.w = w;
        p.tau = tau;
        p.F0 = F0;
        p.Fold = F[cur];
        p.Fnew = F[1 - cur];
        p.maxdiff = d_max;
        prof_mark(c, PGB_PROF_COLLISION);
        k_bte_iter<<<(unsigned)c->nrows_active, kIterThreads, 0, c->stream>>>(p);
        prof_mark(c, PGB_PROF_COLLISION);
        PGB_LAUNCH_CHECK(c);
        unsigned long long hm = 0;
        PGB_CUDA_TRY(c, cudaMemcpyAsync(&hm, d_max, 8, cudaMemcpyDeviceToHost, c->stream));
        PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cur = 1 - cur;
        ++it;
        double diff;
        std::memcpy(&diff, &hm, 8);
        if (diff <= tol * f0max) break;
    }
    if (iters_out) *iters_out = it;
    if ((st = mobility_sum(c, d_win, mu, v, F[cur], mob, &nsum)) != PGB_OK) return st;
    if (d_F) PGB_CUDA_TRY(c, cudaMemcpyAsync(d_F, F[cur], 24 * (size_t)ns, cudaMemcpyDeviceToDevice, c->stream));
    if (d_tau) PGB_CUDA_TRY(c, cudaMemcpyAsync(d_tau, tau, 8 * (size_t)ns, cudaMemcpyDeviceToDevice, c->stream));
    PGB_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PGB_OK;
}

}  // namespace pgb
