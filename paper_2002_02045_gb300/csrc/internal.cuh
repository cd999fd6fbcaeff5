// Internal declarations shared by the translation units of libpertgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pertgb.h"

// ---------------------------------------------------------------------------
// physical constants (CODATA 2018)
// ---------------------------------------------------------------------------
namespace pgb {
constexpr double kHbarEvS = 6.582119569e-16;     // eV s
constexpr double kBoltzEvK = 8.617333262e-5;     // eV / K
constexpr double kAmuKg = 1.66053906660e-27;     // kg
constexpr double kBohrM = 0.529177210903e-10;    // m
constexpr double kEvJ = 1.602176634e-19;         // J
// (hbar w)^2 [eV^2] = kOmega2 * lambda for lambda in eV/(bohr^2 amu); the same
// number divided by 2 M[amu] hbar w[eV] is the squared zero-point length in bohr^2.
constexpr double kOmega2 = kHbarEvS * kHbarEvS * kEvJ / (kAmuKg * kBohrM * kBohrM);
constexpr double kOmegaMinEv = 1e-4;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kTwoPiOverHbar = 2.0 * kPi / kHbarEvS;
constexpr double kFemto = 1e-15;
constexpr double kDeltaCut = 7.0;                // |x|/sigma beyond which a term is skipped
constexpr double kHartreeEv = 27.211386245988;   // eV; e^2 / (4 pi eps_0) = 1 hartree bohr
constexpr double kEwaldCut = 40.0;               // Ewald terms with (q+G).eps.(q+G)/(4 Lambda) above this are dropped
constexpr int kMaxNw = 16;
constexpr int kMaxNmode = 15;
}  // namespace pgb

namespace pgb {
// Real cos/sin form of a Hermitian Fourier sum X(k) = sum_R e^{ik.R} X(R) over
// one representative R of each {R, -R}: rows 2r (cos) and 2r+1 (sin) of T hold
// the packed upper triangle (n real diagonal entries, then (re, im) of (i, j),
// i < j, row by row) of C_R and S_R.
struct HermTab {
    int n = 0, nrep = 0, M = 0;   // matrix size, representatives, max |R_d|
    int32_t *d_R = nullptr;       // [nrep][3]
    double *d_T = nullptr;        // [2 nrep][n*n]
    float2 *d_T2 = nullptr;       // the same split into (hi, lo) floats
};
}  // namespace pgb

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct pgb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;

    // model
    bool has_model = false;
    int nw = 0, nat = 0, nm = 0;
    int nRH = 0, nRD = 0, nRge = 0, nRgp = 0;
    std::vector<double> mass;
    int32_t *d_RH = nullptr, *d_RD = nullptr, *d_Rge = nullptr, *d_Rgp = nullptr;
    double2 *d_H = nullptr;      // [nRH][nw*nw]
    pgb::HermTab htH;            // cos/sin form of H(k) (bands_mixed.cu)
    double2 *d_D = nullptr;      // [nRD][nm*nm] (imaginary part 0)
    double *d_mode_scale = nullptr;  // [nm] 1/sqrt(M_kappa) per ka
    pgb::HermTab htD;            // cos/sin form of the mass-scaled D(q)
    double2 *d_g64 = nullptr;    // [nRge][nRgp*nm*nw*nw]
    float2 *d_g32 = nullptr;
    int nKp = 0;                 // rows of the R_p sum: nRgp, plus nm long-range rows for polar models

    // lattice (pgb_set_lattice) and long-range polar coupling (pgb_set_polar)
    bool has_lattice = false;
    double lat[9] = {0};         // rows a_i, bohr
    double rec[9] = {0};         // rows b_i, 1/bohr (a_i . b_j = 2 pi delta_ij)
    double omega = 0.0;          // cell volume, bohr^3
    std::vector<double> tau;     // [nat][3] bohr
    std::vector<double> zstar;   // [nat][3][3]
    double2 *d_Hd = nullptr;     // [nRH][3][nw][nw] i R^a H(R), eV bohr (band velocities)
    bool polar = false;
    double eps_inf[9] = {0};
    double ewald_lambda = 0.0;
    double *d_polar = nullptr;   // tau [nat][3] then Z* [nat][3][3]
    int32_t *d_gvec = nullptr;   // [nG][3] integer G candidates of the Ewald sum
    int nG = 0;
    double2 *d_polarL = nullptr; // [Nq][nm] long-range term on the q grid

    // grids
    bool has_grids = false;
    int kg[3] = {0, 0, 0}, qg[3] = {0, 0, 0};
    int64_t Nk = 0, Nq = 0;
    double eps_ref = 0.0;        // band-energy shift of the FP32 (hi, lo) energy tables
    double *d_eps = nullptr;     // [Nk][nw]
    double2 *d_U = nullptr;      // [Nk][nw][nw], U[i][n]
    float2 *d_U32 = nullptr;
    float2 *d_U32T = nullptr;    // [n][i][Nk] FP32, grid index fastest (fused tensor-core epilogue)
    double *d_hw = nullptr;      // [Nq][nm]
    double2 *d_coef = nullptr;   // [Nq][nm(nu)][nm(ka)] zero-point-scaled eigenvectors
    float2 *d_coef32 = nullptr;
    float2 *d_coefT = nullptr;   // [nu][ka][Nq] FP32, grid index fastest (fused tensor-core epilogue)
    double2 *d_phq64 = nullptr;  // [Nq][nRgp] exp(i q.Rp), built on first use
    float2 *d_phq32 = nullptr;
    void *d_asplit = nullptr;    // [4][Nq][Kp] hi/lo split phases for the tensor-core q-sum
    int asplit_prec = -1;        // precision the split was built for
    void *d_gsplit = nullptr;    // [4][nRgp*nm*nw*nw][Kp(nRge)] hi/lo split g~, B of the tensor-core R_e sum
    int gsplit_prec = -1;
    int *d_err = nullptr;        // device error word of the tensor-core kernels

    // collision list
    bool has_coll = false;
    int64_t nstates = 0, nnz = 0;
    int band_lo = 0, band_hi = 0;
    double *d_eps_state = nullptr;   // [nstates]
    int64_t *d_rowptr = nullptr;     // [nstates+1]
    int32_t *d_col = nullptr;        // [nnz]
    float *d_a = nullptr, *d_b = nullptr;
    double *d_rowsum_a = nullptr;    // [nstates]
    int32_t *d_active_rows = nullptr;   // non-empty rows
    int64_t nrows_active = 0;
    double *d_f[4] = {nullptr, nullptr, nullptr, nullptr};  // RK4 stage buffers
    float *d_f32[3] = {nullptr, nullptr, nullptr};          // FP32 copies gathered by the collision kernel
    int32_t *d_coo_row = nullptr, *d_coo_col = nullptr, *d_coo_mode = nullptr;  // the list as given or built
    float *d_coo_g2 = nullptr;
    double coll_T = 0.0, coll_sigma = 0.0;
    int coll_nb = 0;
    double coll_elo = -1e300, coll_ehi = 1e300;   // energy window of the list's states

    // transposed list for the reverse-mode pass, built on first use
    bool adj_ready = false;
    int64_t *d_t_colptr = nullptr;   // [nstates+1] entries with col == c
    int32_t *d_t_src = nullptr;      // [nnz] row of each transposed entry
    int32_t *d_t_eidx = nullptr;     // [nnz] its index in the list
    float *d_t_a = nullptr, *d_t_b = nullptr;           // a, b of the list
    float *d_t_alpha = nullptr, *d_t_beta = nullptr;    // a / |g|^2, b / |g|^2
    int32_t *d_t_active = nullptr;   // columns with entries
    int64_t t_nactive = 0;

    // scratch (grown on demand, freed in destroy)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;

    // kernel timing with CUDA events on the context's stream (pgb_profile)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev[PGB_PROF_NKERNELS];   // start, stop, start, stop, ...
    double prof_ms[PGB_PROF_NKERNELS] = {0};
    int64_t prof_n[PGB_PROF_NKERNELS] = {0};
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define PGB_CUDA_TRY(ctx, expr)                                                        \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) {                                                       \
            (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(_e);           \
            return _e == cudaErrorMemoryAllocation ? PGB_ENOMEM : PGB_ECUDA;           \
        }                                                                              \
    } while (0)

#define PGB_LAUNCH_CHECK(ctx)                                                          \
    do {                                                                               \
        (ctx)->launches++;                                                             \
        cudaError_t _e = cudaGetLastError();                                           \
        if (_e != cudaSuccess) {                                                       \
            (ctx)->err = std::string("kernel launch: ") + cudaGetErrorString(_e);      \
            return PGB_ECUDA;                                                          \
        }                                                                              \
    } while (0)

namespace pgb {

// Every device allocation of the library goes through these calls (never
// cudaMalloc / cudaMallocAsync directly): they count allocations and can be
// told by pgb_diag_fail_alloc to refuse one on the host, as an out-of-memory
// device would, so that each caller's PGB_ENOMEM path can be exercised.
cudaError_t dev_malloc_raw(void **p, size_t bytes, cudaStream_t stream, bool async);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes, nullptr, false);
}
template <typename T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t stream) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes, stream, true);
}

pgb_status ensure_scratch(pgb_ctx *c, size_t bytes);
// Bracket one launch of a timed kernel class with events (no-op unless enabled).
void prof_mark(pgb_ctx *c, int id);
template <typename T>
pgb_status dalloc(pgb_ctx *c, T **p, size_t count) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) return PGB_OK;
    PGB_CUDA_TRY(c, dev_malloc((void **)p, count * sizeof(T)));
    return PGB_OK;
}
template <typename T>
void dfree(T **p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

// interpolation kernels (interp.cu)
pgb_status launch_phase_grid(pgb_ctx *c, const int grid[3], const int32_t *d_idx, int64_t npts,
                             const int32_t *d_R, int nR, void *out, bool fp32, int64_t ld = 0);
pgb_status launch_phase_pts(pgb_ctx *c, const double *d_pts, int64_t npts, const int32_t *d_R, int nR,
                            void *out, bool fp32, int64_t ld = 0);

// long-range polar coupling (polar.cu)
pgb_status polar_grid_table(pgb_ctx *c);
// q tables [npts][nKp]: e^{iq.Rp} for the nRgp lattice vectors, then the long-range columns
pgb_status launch_qtable_grid(pgb_ctx *c, const int32_t *d_idx, int64_t npts, void *out, bool fp32);
pgb_status launch_qtable_pts(pgb_ctx *c, const double *d_pts, int64_t npts, void *out, bool fp32);
pgb_status launch_ewald_pts(pgb_ctx *c, const double *d_pts, int64_t npts, void *out, int64_t ld, int col0,
                            bool fp32);
std::vector<int32_t> ewald_candidates(const double lat[9], const double eps[9], double lambda);

// Monte-Carlo q rates and tetrahedron populations (mcq.cu); device pointers
pgb_status launch_mc_qpoints(pgb_ctx *c, int64_t nq, const double *u, int sampling, double width, double *q,
                             double *pinv);
pgb_status launch_mc_epilogue(pgb_ctx *c, bool fp32, int64_t nkb, int64_t nq, const void *C, int64_t ldc,
                              const void *Ukq, const double *eps_k, const double *eps_kq, const double *hw,
                              const void *coef, const double *pinv, double T, double mu, double sigma, double *partial,
                              double *acc);
int64_t mc_partial_count(const pgb_ctx *c, int64_t nkb, int64_t nq);
pgb_status launch_mc_finish(pgb_ctx *c, int64_t nk, int64_t nq, double sigma, const double *acc, double *gamma,
                            double *err);
pgb_status launch_population(pgb_ctx *c, const double *f, const double *E, int64_t nE, double *out);

// band velocities and transport (transport.cu); device pointers
pgb_status build_velocity_tables(pgb_ctx *c);
pgb_status band_velocities(pgb_ctx *c, const int32_t *d_kidx, int64_t nk, double *d_v);
pgb_status transport(pgb_ctx *c, double mu, int precision, int max_iter, double tol, double *mob_rta, double *mob,
                     int64_t *iters_out, double *d_F, double *d_tau);
pgb_status launch_cgemm(pgb_ctx *c, bool fp32, int64_t batch, int64_t M, int64_t N, int64_t K,
                        const void *A, int64_t lda, int64_t strideA, const void *B, int64_t ldb,
                        int64_t strideB, void *C, int64_t ldc, int64_t strideC);
pgb_status launch_heevj(pgb_ctx *c, int64_t count, int n, double2 *d_mat, const double *d_scale,
                        double *d_eval, double2 *d_evec);
// band interpolation for the FP32 paths (bands_mixed.cu)
pgb_status build_herm_table(pgb_ctx *c, HermTab *t, const int32_t *R, const double *X, int nR, int n);
void free_herm_table(HermTab *t);
pgb_status launch_herm_sum(pgb_ctx *c, const HermTab &t, const double *d_pts, int64_t np, double *d_out);
pgb_status launch_heev_mixed(pgb_ctx *c, int64_t count, int n, const double *d_Hp, double *d_eval, float2 *d_U32,
                             double2 *d_U64, bool refine_vectors);
pgb_status launch_phonon_coef(pgb_ctx *c, int64_t nq, int nm, const double *d_eval,
                              const double2 *d_evec, const double *d_mode_scale, double *d_hw,
                              double2 *d_coef);
pgb_status launch_to_f32(pgb_ctx *c, const double2 *src, float2 *dst, int64_t n);
pgb_status launch_fold_u(pgb_ctx *c, bool fp32, int64_t nb, const int32_t *d_kidx, int nRgp, int nm,
                         int nw, const void *S1, const void *U, void *G);
struct RatesArgs {
    int64_t nb;            // k points in this batch
    const int32_t *kidx;   // [nb] k-grid indices (device)
    int64_t Nq;
    int kg[3], qg[3];
    int nw, nm;
    const void *C;         // [nb][Nq][nm*nw*nw] Wannier-gauge g with U(k) folded
    const void *U;         // [Nk][nw][nw]
    const void *coef;      // [Nq][nm][nm]
    const double *eps;     // [Nk][nw]
    const double *hw;      // [Nq][nm]
    double T, mu, sigma;
    const float *eps32;    // [Nk][nw] screening copy
    const double *focc;    // [Nk][nw] Fermi-Dirac occupations
    const double *nbe;     // [Nq][nm] Bose-Einstein occupations
    const float *hw32;     // [Nq][nm]
    double *partial;       // [nb][nqblk][nm][nw]
    int64_t nqblk;
    int qpb;               // q per block and iteration
    int qiters;            // iterations per block
};
pgb_status launch_occ_tables(pgb_ctx *c, double T, double mu, double *focc, float *eps32, double *nbe,
                             float *hw32);
pgb_status launch_rates_epilogue(pgb_ctx *c, bool fp32, const RatesArgs &a);
pgb_status launch_rates_reduce(pgb_ctx *c, int64_t nb, int64_t nqblk, int nm, int nw, double scale,
                               const double *partial, double *gamma, double *gamma_mode);
struct GArgs {
    int64_t nk, nq;
    int nw, nm;
    const void *C;         // [nk][nq][ldc]: columns (n, ka, i) of nm*nw*nw, then padding
    int64_t ldc;           // column stride of C (>= nm*nw*nw)
    const void *Ukq;       // [nk*nq][nw][nw]
    const void *coef;      // [nq][nm][nm]
    int out_mode;
    double *out;
};
pgb_status launch_g_epilogue(pgb_ctx *c, bool fp32, const GArgs &a);
pgb_status launch_g_abs(pgb_ctx *c, int64_t npairs, int nm, int nw, const double *full, double *out);
pgb_status launch_kplusq_pts(pgb_ctx *c, const double *d_k, int64_t nk, const double *d_q, int64_t nq,
                             double *d_kq);
pgb_status launch_window(pgb_ctx *c, const double *d_eps, int64_t Nk, int nw, double lo, double hi,
                         int32_t *d_flag);

// tensor-core q-sum (tc_qsum.cu)
int tc_kpad(int nR);
bool tc_supported(int ncol);
pgb_status launch_split_phases(pgb_ctx *c, bool tf32, const int grid[3], int64_t Nq, const int32_t *d_R, int nR,
                               int Kp, void *out, const double2 *L = nullptr, int nL = 0);
pgb_status launch_split_phases_pts(pgb_ctx *c, bool tf32, const int grid[3], const int32_t *d_pts, int64_t n,
                                   const int32_t *d_R, int nR, int Kp, void *out);
pgb_status launch_split_gT(pgb_ctx *c, bool tf32, int nR, int64_t ncol, int Kp, const double2 *g, void *out);
pgb_status launch_split_table(pgb_ctx *c, bool tf32, int64_t n, int ncols, int64_t ld, int Kp, const double2 *T,
                              void *out);
pgb_status launch_split_g(pgb_ctx *c, bool tf32, int64_t nb, int nR, int ncol, int Kp, const void *G, void *out,
                          int ncol_pad = 0);
pgb_status launch_split_g6(pgb_ctx *c, bool tf32, int64_t nb, int nR, int ncol, int Kp, const void *G, void *out);
// C[b][q][c] for q < Nq from rows q_off .. q_off + Nq of an A table of nqA rows (nqA <= 0: Nq)
pgb_status launch_tc_qsum(pgb_ctx *c, bool tf32, int64_t nb, int64_t Nq, int ncol, int Kp, void *Asplit,
                          void *Bsplit, float2 *C, int *d_err, int64_t nqA = 0, int64_t q_off = 0);
pgb_status tc_qsum_prepare(pgb_ctx *c, bool tf32);

// warp-per-row rates epilogue over a q slab of tensor-core q-sums (rates_warp.cu)
struct WarpRatesArgs {
    int nw, nm, ib;        // ib: lanes per mode column of a row (warp_rates_ib)
    int kg[3], qg[3];
    int64_t q_off, nqs;    // q-grid index of the slab's first row, rows in the slab
    int qc, nch;           // q-points per task, tasks per k in the slab
    int64_t nb;            // k-points of the batch
    const float2 *C;       // [nb][nqs][ldc] R_p sums, columns (n, ka, i)
    int64_t ldc;
    const int32_t *kidx;   // [nb] k-grid indices
    const double *eps;     // [Nk][nw]
    const float *eps32;    // [Nk][nw]
    const float2 *U;       // [Nk][i][m] FP32
    const float2 *coef;    // [Nq][nu][ka] FP32
    const double *hw;      // [Nq][nm]
    const float *hw32;     // [Nq][nm]
    const double *focc;    // [Nk][nw]
    const double *nbe;     // [Nq][nm]
    double sigma;
    double *partial;       // [nb][nqblk][nm][nw]; this slab writes blocks blk0 .. blk0 + nch
    int64_t nqblk, blk0;
};
int warp_rates_ib(int nw, int nm);
pgb_status launch_rates_warp(pgb_ctx *c, const WarpRatesArgs &a);

// fused tensor-core rates (tc_rates.cu)
struct FusedLaunch {
    int64_t nb;
    const int32_t *kidx;
    int Kp;
    void *Bsplit;
    const float2 *ehl;     // [nw][Nk] (e - e_ref) as hi + lo floats
    const float *focc32;   // [nw][Nk]
    const float2 *whl;     // [nm][Nq] hbar*omega as hi + lo floats
    const float *nbe32;    // [nm][Nq]
    double sigma;
    double *partial;   // [nb][ceil(Nq/128)][nm][nw]
};
pgb_status launch_fp32_tables(pgb_ctx *c, const double *focc, const double *nbe, float2 *ehl, float *focc32,
                              float2 *whl, float *nbe32);
bool tc_fused_supported(int nw, int nm);
pgb_status launch_tc_rates(pgb_ctx *c, bool tf32, const FusedLaunch &L);
pgb_status diag_delta_weights(pgb_ctx *c, int64_t n, const double *en, const double *em, const double *hw,
                              double eps_ref, double sigma, float *out);
pgb_status launch_transpose_u(pgb_ctx *c);
pgb_status launch_transpose_coef(pgb_ctx *c);

// scattering list from the grid (list.cu)
struct ListLaunch {
    int64_t nb;
    const int32_t *kidx;
    int64_t na;             // k-points holding a window state
    const int32_t *win;     // [na] their grid indices (the k' = k + q of the restricted sum)
    int band_lo, nbnd;
    const uint8_t *inwin;
    double cut;
};
pgb_status list_count(pgb_ctx *c, const ListLaunch &L, unsigned long long *d_counter);
pgb_status list_gather_qrows(pgb_ctx *c, const ListLaunch &L, const void *phq, void *out);
pgb_status list_fill(pgb_ctx *c, const ListLaunch &L, const void *C, unsigned long long *d_counter, uint64_t *keys,
                     float *vals, unsigned long long cap);
pgb_status list_sort_decode(pgb_ctx *c, int64_t n, int ns, uint64_t *keys, float *vals, uint64_t *keys_alt,
                            float *vals_alt, int32_t *row, int32_t *col, int32_t *mode, float *g2);

// collision kernels (collision.cu)
pgb_status launch_coll_coeffs(pgb_ctx *c, double T, double sigma, const int32_t *row, const int32_t *col,
                              const int32_t *mode, const float *g2, int64_t nnz, int nb);
pgb_status launch_collision(pgb_ctx *c, const double *f, const float *f32, double *I, int stage, double dt,
                            double *acc, double *fnext, float *fnext32, const double *fbase, double *D = nullptr);
pgb_status launch_coll_values(pgb_ctx *c, const int32_t *row, const int32_t *col, const int32_t *mode,
                              const float *g2, int64_t nnz);
pgb_status launch_coll_rowsum(pgb_ctx *c);
void free_adjoint(pgb_ctx *c);
pgb_status adjoint_values_changed(pgb_ctx *c);   // a, b of the list were recomputed

// reverse-mode derivatives of the collision integral and RK4 (adjoint.cu); device pointers
pgb_status collision_vjp(pgb_ctx *c, const double *f, const double *lam, double *out_f, double *out_g2);
pgb_status rk4_adjoint(pgb_ctx *c, const double *f0, double dt_fs, int64_t nsteps, int64_t ckpt,
                       const double *lam_end, double *lam0, double *dg2, double *f_end);
pgb_status launch_f64_to_f32(pgb_ctx *c, const double *x, float *y, int64_t n);

}  // namespace pgb
