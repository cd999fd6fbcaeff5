/*
 * pertgb.h - C ABI of the GB300 e-ph hot path (Perturbo method, arXiv 2002.02045).
 *
 * The library evaluates, on one CUDA GPU:
 *   - Wannier interpolation of bands and phonons       (Sec. 2.2.1 Eq. wannier_3; Sec. 2.2.2 Eq. IFC2)
 *   - e-ph matrix elements g_mn nu(k,q)                 (Sec. 2.2.3 Eqs. eph_mat_wann2, eph_mat, g_abs)
 *   - RTA scattering rates Gamma_nk                     (Sec. 2.1.2 Eqs. scatter_rate, BTE_W)
 *   - the e-ph collision integral I[f]_nk               (Sec. 2.1 Eq. e_ph_scattering)
 *   - explicit RK4 time stepping of df/dt = I[f]        (Sec. 2.1.1)
 *
 * Conventions (every entry point):
 *   - k, q are crystal coordinates (units of the reciprocal vectors); R are
 *     integer crystal coordinates; the Fourier phase is exp(2 pi i k.R).
 *   - Complex arrays are interleaved (re, im) in the stated real type.
 *   - Energies and hbar*omega in eV, D(R) in eV/bohr^2, masses in amu,
 *     g~(Re,Rp) in eV/bohr, temperatures in K, rates and I[f] in 1/s, time
 *     steps in fs.  Gaussian delta: exp(-x^2/s^2)/(s sqrt(pi)).  Modes with
 *     hbar*omega < 1e-4 eV carry no weight.  1/N_q is the q-grid size.
 *   - Grids are Gamma-centred Monkhorst-Pack: point p = (i1*n2 + i2)*n3 + i3
 *     is (i1/n1, i2/n2, i3/n3).  The q grid must divide the k grid.
 *   - Band index n is the initial state at k, m the final state at k+q.
 *   - Buffers marked "host or device" may be either: device pointers are used
 *     in place (stream-ordered, no synchronisation); host pointers are copied
 *     through the context's stream and the call synchronises before returning.
 *   - Caller owns every buffer it passes; the library owns the copies it makes
 *     in set_model / set_grids / build_collision and frees them in destroy.
 *   - Errors return a negative pgb_status and leave outputs unwritten for
 *     argument errors; pgb_last_error() gives a message.  No call traps the
 *     GPU, and there is no CPU fallback: without a usable CUDA device every
 *     call returns PGB_ECUDA.
 */
#ifndef PERTGB_H
#define PERTGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pgb_ctx pgb_ctx;

typedef enum {
    PGB_OK = 0,
    PGB_EINVAL = -1,    /* bad argument, shape or unsupported mode            */
    PGB_ESTATE = -2,    /* call order violated (e.g. rates before set_grids)   */
    PGB_ENOMEM = -3,    /* device allocation failed                            */
    PGB_ECUDA = -4,     /* CUDA runtime error                                  */
    PGB_ETIMEOUT = -5,  /* a bounded device wait ran out                       */
} pgb_status;

typedef enum {
    PGB_FP64 = 0,        /* every step in FP64                                       */
    PGB_FP32 = 1,        /* Fourier sums and rotations in FP32 SIMT, energies FP64   */
    PGB_TC_TF32X3 = 2,   /* q-sum on tcgen05 kind::tf32, 3-product hi/lo split        */
    PGB_TC_BF16X3 = 3,   /* q-sum on tcgen05 kind::f16 (bf16), 3-product hi/lo split  */
} pgb_precision;

typedef enum {
    PGB_G2_FULL = 0,     /* out[k][q][nu][m][n] = |g_mn nu(k,q)|^2, double, eV^2      */
    PGB_G_ABS = 1,       /* out[k][q][nu] = |g_nu(k,q)| of Eq. g_abs, double, eV      */
} pgb_g_output;

/* Real-space model (all host pointers, copied by pgb_set_model).
 * H(R): Eq. wannier_3 input, H[r][n][n'] = <n 0|H|n' R_r>, H(-R) = H(R)^dagger.
 * D(R): Eq. IFC2 input without mass factor, D[r][ka][k'b] real, ka = 3 kappa + alpha.
 * g~(Re,Rp): Eq. eph_mat_wann2 input on the dense product of two R lists,
 *            g[re][rp][ka][i][j], complex64 (g_is_double = 0) or complex128.   */
typedef struct {
    int nw;                    /* Wannier functions (bands)          */
    int nat;                   /* atoms; nmode = 3 nat               */
    const double *mass;        /* [nat] amu                          */
    int nR_H;
    const int32_t *R_H;        /* [nR_H][3]                          */
    const double *H;           /* [nR_H][nw][nw] complex128          */
    int nR_D;
    const int32_t *R_D;        /* [nR_D][3]                          */
    const double *D;           /* [nR_D][3nat][3nat] real            */
    int nR_ge;
    const int32_t *R_ge;       /* [nR_ge][3]                         */
    int nR_gp;
    const int32_t *R_gp;       /* [nR_gp][3]                         */
    const void *g;             /* [nR_ge][nR_gp][3nat][nw][nw]       */
    int g_is_double;
} pgb_model;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream); every launch of the context goes there. */
pgb_status pgb_create(pgb_ctx **out, int device, void *cuda_stream);
void pgb_destroy(pgb_ctx *ctx);
const char *pgb_last_error(const pgb_ctx *ctx);
const char *pgb_status_string(int status);

/* Copy the model to the device.  Checks: sizes > 0, nw <= 16, nat <= 5,
 * finite values, H(-R) = H(R)^dagger and D(-R) = D(R)^T to 1e-10 (both R
 * lists must be closed under inversion).  Returns PGB_EINVAL otherwise.      */
pgb_status pgb_set_model(pgb_ctx *ctx, const pgb_model *model);

/* Fix the k and q grids.  Computes eps_nk and U(k) on every k-grid point
 * (Eq. wannier_3) and hbar*omega_nu q, e_nu q on every q-grid point (Eq. IFC2),
 * in FP64 with a cyclic complex Jacobi eigensolver (ascending order).
 * Each q-grid size must divide the k-grid size along the same axis.          */
pgb_status pgb_set_grids(pgb_ctx *ctx, const int kgrid[3], const int qgrid[3]);

/* Lattice of the model (Sec. 2.2): lattice[9] rows a_1, a_2, a_3 in bohr
 * (Cartesian), tau [nat][3] atom positions in bohr (host pointers, copied).
 * R vectors stay integer crystal coordinates (R = n_1 a_1 + n_2 a_2 + n_3 a_3).
 * Needed by pgb_band_velocities, pgb_transport and pgb_set_polar; reset by
 * pgb_set_model.  Re-applies an active polar term with the new positions.   */
pgb_status pgb_set_lattice(pgb_ctx *ctx, const double lattice[9], const double *tau);

/* Long-range (Froehlich) coupling of polar materials (Sec. 2.2.4, Eqs.
 * e_ph_long, smooth_phase).  zstar [nat][3][3] Born effective charges with
 * [(q+G).Z*_k]_a = sum_b (q+G)_b zstar[k][b][a]; eps_inf[9] the symmetric
 * positive-definite high-frequency dielectric tensor; lambda the Ewald
 * parameter Lambda (1/bohr^2).  In the Wannier gauge the term is
 *   L^{ka}(q) = i (e^2/(eps_0 Omega)) sum_{G, q+G != 0} [(q+G).Z*_k]_a e^{-i tau_k.(q+G)}
 *               e^{-(q+G).eps.(q+G)/(4 Lambda)} / ((q+G).eps.(q+G))   (eV/bohr),
 * over every G with (q+G).eps.(q+G)/(4 Lambda) <= 40, and g~ gains
 * L^{ka}(q) delta_ij, so that g_mn nu(k,q) gains
 * sqrt(hbar/2 omega) sum_ka e^{ka}_nu/sqrt(M_k) L^{ka}(q) [U^dagger(k+q) U(k)]_mn in
 * every later pgb_interpolate_g, pgb_scattering_rates(_noalloc) and
 * pgb_build_collision_grid (a list built before keeps its |g|^2).  zstar
 * NULL removes the term.  Host pointers, copied.  Needs pgb_set_lattice.     */
pgb_status pgb_set_polar(pgb_ctx *ctx, const double *zstar, const double eps_inf[9], double lambda);

/* L^{ka}(q) of pgb_set_polar at qpts [nq][3] (crystal coordinates, host or
 * device): out [nq][nmode] complex as (re, im) doubles, eV/bohr (host or
 * device).  Zero without a polar term.                                        */
pgb_status pgb_long_range_g(pgb_ctx *ctx, const double *qpts, int64_t nq, double *out);

/* Read the grid quantities computed by set_grids (host or device outputs).
 * eps [Nk][nw] eV; hw [Nq][nmode] eV.  Either pointer may be NULL.           */
pgb_status pgb_get_grid_energies(pgb_ctx *ctx, double *eps, double *hw);

/* Energy window (Sec. 4.3): list the k-grid points that have at least one
 * band in [e_lo, e_hi].  k_idx_out (host or device, capacity Nk) receives
 * the ascending point indices, *n_out their count.                           */
pgb_status pgb_window(pgb_ctx *ctx, double e_lo, double e_hi, int32_t *k_idx_out, int64_t *n_out);

/* e-ph matrix elements at arbitrary points (Eqs. eph_mat_wann2, eph_mat).
 * kpts [nk][3], qpts [nq][3] (host or device, crystal coordinates).  Bands at
 * k, k+q and phonons at q are interpolated for the call.  precision: PGB_FP64
 * or PGB_FP32.  out (host or device): see pgb_g_output, always double.        */
pgb_status pgb_interpolate_g(pgb_ctx *ctx, const double *kpts, int64_t nk, const double *qpts,
                             int64_t nq, int precision, int out_mode, double *out);

/* RTA scattering rates (Eqs. scatter_rate, BTE_W) for the k-grid points
 * k_idx[0..nk) (host or device) and every band, summing q over the whole q
 * grid, m over every band and nu over every mode.  f0 is Fermi-Dirac at (T,
 * mu), N0 Bose-Einstein at T.  Terms with |x|/sigma > 7 (x the energy
 * mismatch) are skipped: each is below exp(-49) of a peak term.
 * gamma_out [nk][nw] (host or device, 1/s); gamma_mode_out [nk][nmode][nw]
 * or NULL.                                                                    */
pgb_status pgb_scattering_rates(pgb_ctx *ctx, const int32_t *k_idx, int64_t nk, double T_K,
                                double mu_eV, double sigma_eV, int precision, double *gamma_out,
                                double *gamma_mode_out);

/* Scattering list for the collision integral (Sec. 4.3 (k,q) pairs;
 * Eq. e_ph_scattering).  States are s = ik*nb + (n - band_lo) for every
 * k-grid point ik and n in [band_lo, band_hi); the q grid must equal the k
 * grid.  Each entry e (host or device arrays, rows non-decreasing) is the
 * term s = row[e] -> s' = col[e] by mode mode[e] with |g|^2 = g2[e] (eV^2);
 * q is the k-grid difference k(s') - k(s).  For each entry the library
 * computes, in FP64, a = (2pi/hbar)(1/Nq)|g|^2 [d_em (N+1) + d_abs N] and
 * b = (2pi/hbar)(1/Nq)|g|^2 [d_em N + d_abs (N+1)] with d_em = delta(e_s - hw - e_s'),
 * d_abs = delta(e_s + hw - e_s'), stores them as FP32 in a CSR list, and
 * later evaluates I_s = sum_e [ -f_s (1 - f_s') a_e + f_s' (1 - f_s) b_e ].   */
pgb_status pgb_build_collision(pgb_ctx *ctx, int band_lo, int band_hi, double T_K, double sigma_eV,
                               int64_t nnz, const int32_t *row, const int32_t *col,
                               const int32_t *mode, const float *g2);

/* Scattering list built on the device from the model (Sec. 4.3): states
 * s = ik*nb + (n - band_lo) for every k-grid point and n in [band_lo,
 * band_hi) (q grid = k grid); only states with e_lo <= eps <= e_hi take part
 * (the others keep empty rows).  For every (k, q) with both states in the
 * window and every mode, the term is kept when |x_em| or |x_abs| is at most
 * 7 sigma; |g_mn nu(k,q)|^2 comes from the FP32 interpolation (Eqs.
 * eph_mat_wann2, eph_mat).  Each unordered process is evaluated once (s <=
 * s') and written to both rows with the same |g|^2, so sum_s I_s = 0 to
 * rounding.  Entries are ordered by (row, col, mode).  Then proceeds as
 * pgb_build_collision.  *nnz_out (may be NULL) receives the entry count.     */
pgb_status pgb_build_collision_grid(pgb_ctx *ctx, int band_lo, int band_hi, double e_lo, double e_hi, double T_K,
                                    double sigma_eV, int64_t *nnz_out);

/* Copy out the current list (as given to pgb_build_collision, or as built by
 * pgb_build_collision_grid, with |g|^2 as last set): row, col, mode int32
 * and |g|^2 float32, [nnz] each (host or device; any may be NULL).           */
pgb_status pgb_collision_list(pgb_ctx *ctx, int32_t *row, int32_t *col, int32_t *mode, float *g2);

/* State energies of the collision list [nstates] (host or device).          */
pgb_status pgb_collision_energies(pgb_ctx *ctx, double *eps_state, int64_t *nstates_out);

/* I[f] (Eq. e_ph_scattering) for f [nstates] -> I_out [nstates], 1/s.       */
pgb_status pgb_collision(pgb_ctx *ctx, const double *f, double *I_out);

/* nsteps explicit RK4 steps (Sec. 2.1.1) of df/dt = I[f], step dt_fs, in place. */
pgb_status pgb_step_rk4(pgb_ctx *ctx, double *f, double dt_fs, int64_t nsteps);

/* Band velocities (Eqs. velocity, wannier_4) at the k-grid points k_idx[0..nk)
 * (host or device): v_out [nk][nw][3] in m/s (host or device), with
 * hbar v^a_nk = [U^dagger(k) H_a(k) U(k)]_nn, H_a(k) = sum_R e^{ik.R} H(R) i R^a,
 * R^a Cartesian, in FP64.  For bands degenerate within 1e-6 eV the velocities
 * along each direction are the ascending eigenvalues of that direction's
 * matrix restricted to the degenerate subspace.  Needs set_lattice, set_grids. */
pgb_status pgb_band_velocities(pgb_ctx *ctx, const int32_t *k_idx, int64_t nk, double *v_out);

/* Mobility from the linearised BTE (Sec. 2.1.2: Eqs. BTE_lin, BTE_iter, BTE_W,
 * cond) on the current collision list, over its states inside its energy
 * window (all states for a list given to pgb_build_collision), at the list's
 * T and sigma and chemical potential mu_eV:
 *   tau_nk = 1/Gamma_nk from pgb_scattering_rates over the whole q grid, every
 *     final band and mode, in `precision` (states with Gamma = 0 get tau = 0);
 *   v_nk from pgb_band_velocities;
 *   W_e = (2 pi/hbar)(1/N_q)|g|^2 [d(e_s - hw - e_s')(1 + N - f0_s') + d(e_s + hw - e_s')(N + f0_s')]
 *     per list entry;
 *   F^0 = tau v, F^{i+1}_s = tau_s v_s + tau_s sum_{e in row s} W_e F^i_{col e}, until
 *     max |F^{i+1} - F^i| <= tol max |F^0| or max_iter iterations (W, F and
 *     the products in FP64: the iteration matrix's spectral radius is often
 *     within 1e-3 of one, which amplifies any error of W);
 *   mobility[a*3+b] = sum_s v^a_s F^b_s (-df0/de)_s / sum_s f0_s in cm^2/(V s),
 *     -df0/de = f0 (1 - f0)/kT (Eq. cond divided by e n_c, the carriers of
 *     the same states).
 * mobility_rta [9] receives the same with F = F^0 (host or device, both
 * required).  iterations_out (host, may be NULL): iterations run.  F_out
 * [nstates][3] in m and tau_out [nstates] in s (host or device, may be NULL);
 * states outside the window get 0.  Needs set_lattice.                      */
pgb_status pgb_transport(pgb_ctx *ctx, double mu_eV, int precision, int max_iter, double tol,
                         double *mobility_rta, double *mobility, int64_t *iterations_out, double *F_out,
                         double *tau_out);

/* Gamma_nk by Monte-Carlo q sampling (Sec. 4.3: random q in the zone, uniform
 * or Cauchy; Eqs. scatter_rate, BTE_W) at arbitrary points kpts [nk][3]
 * (crystal coordinates, host or device), every band.  The caller supplies the
 * random numbers: u [nq][3] uniforms in [0, 1) (host or device; PGB_EINVAL
 * otherwise), mapped per coordinate to
 *   PGB_Q_UNIFORM: q_i = u_i - 1/2, density p = 1;
 *   PGB_Q_CAUCHY:  q_i = atan(c tan(pi (u_i - 1/2)))/pi, p(q_i) = c/(c^2 cos^2(pi q_i) + sin^2(pi q_i)),
 *                  c = width in (0, 1] (Lorentzian of width ~c/pi about q_i = 0);
 *   Gamma_nk = (1/nq) sum_j y_j, y_j = sum_{m nu} W(k, q_j) / p(q_j),
 * with bands at k + q_j and phonons at q_j interpolated for each sample and g
 * including any polar term.  stderr_out (may be NULL) receives the standard
 * error sqrt(sum_j (y_j - Gamma)^2 / (nq (nq - 1))).  precision: PGB_FP64
 * (everything FP64); PGB_FP32 (FP32 products; bands at k + q_j and phonons at
 * q_j from the cos/sin Fourier sums in double-float and a mixed-precision
 * Jacobi: FP64-refined eigenvalues and phonon modes, FP32 band eigenvectors;
 * energies and weights FP64); PGB_TC_TF32X3 or
 * PGB_TC_BF16X3 (as PGB_FP32, with the R_p sum on the tensor cores in the split
 * precision).  Terms with |x|/sigma > 7 are skipped.  Outputs [nk][nw], 1/s.
 * PGB_ETIMEOUT if a tensor-core pipeline wait ran out (no result).           */
#define PGB_Q_UNIFORM 0
#define PGB_Q_CAUCHY 1
pgb_status pgb_scattering_rates_mc(pgb_ctx *ctx, const double *kpts, int64_t nk, const double *u, int64_t nq,
                                   int sampling, double width, double T_K, double mu_eV, double sigma_eV,
                                   int precision, double *gamma_out, double *stderr_out);

/* Carrier population (Eq. pop) by the linear tetrahedron method on the k grid
 * of the current collision list: for occupations f [nstates] (host or
 * device) and energies E [nE] (eV), N_out [nE] (host or device) receives
 *   N(E) = sum_n (1/V_BZ) int f_n(k) theta(E - e_n(k)) dk   (carriers per cell below E),
 * with e_n and f_n linear on each of the six tetrahedra of every grid cell
 * (cells split along their (0,0,0)-(1,1,1) diagonal), over the list's bands.
 * p(E) integrated over [E_a, E_b) is N(E_b) - N(E_a).                      */
pgb_status pgb_population(pgb_ctx *ctx, const double *f, const double *E, int64_t nE, double *N_out);

/* Batched scattering rates of many independent instances (contexts with
 * their own model and grids, k grid = q grid or commensurate, on one device),
 * in one persistent launch under a captured CUDA graph.
 *
 * pgb_batch_create: ctxs[0..n) (kept by pointer: they must keep their model
 * and grids, and stay alive, while the batch exists); the batch runs on the
 * first context's stream.
 * pgb_batch_rates: for instance i, Gamma_nk (Eqs. scatter_rate, BTE_W; FP32
 * products, FP64 energy differences and weights, terms beyond 7 sigma
 * skipped) of the k-grid points k_idx[i][0..nk[i]) over its whole q grid and
 * every band and mode, at T_K, mu_eV[i] and sigma_eV, into gamma_out[i]
 * [nk[i]][nw_i] (1/s).  k lists and outputs host or device.  Per instance the
 * R_p sums over the whole q grid are formed first (into a [nk][Nq][columns]
 * FP32 buffer of the batch, 8 bytes per entry); one persistent kernel then
 * runs the epilogue of every instance, one unit per (instance, k, q tile)
 * over all its bands.  The first call tunes the block size and the shared-
 * memory budget that sets each instance's q tile (four candidates timed once
 * each); every call with new arguments captures the per-instance set-up
 * (occupations, R_e and R_p sums), the persistent kernel and the reduction
 * into a CUDA graph; calls with the same arguments replay it.  Results do not
 * depend on the schedule.
 * pgb_batch_tuning: the largest per-instance q tile and the block size of the
 * chosen candidate, candidate times (ms, [4], -1 where not run) and graph
 * launches so far (any pointer may be NULL).
 * pgb_batch_set_precision: PGB_FP32 (default: every instance's R_p sum on
 * the CUDA cores, FP32 products) or PGB_TC_BF16X3 / PGB_TC_TF32X3: then every
 * instance takes its R_p sum on the tensor cores (split operands, FP32
 * accumulators, nm*nw*nw columns padded with zeros to a multiple of 96, polar
 * long-range rows included; a tensor-core pipeline time-out returns
 * PGB_ETIMEOUT).  A change drops the captured graph and the tuning.  Error
 * bound against the FP64 oracle: 1e-3 (BF16x3), 1e-5 (TF32x3 and FP32).
 * Other values: PGB_EINVAL.                                                 */
typedef struct pgb_batch pgb_batch;
pgb_status pgb_batch_create(pgb_batch **out, pgb_ctx *const *ctxs, int n);
pgb_status pgb_batch_rates(pgb_batch *batch, const int32_t *const *k_idx, const int64_t *nk, double T_K,
                           const double *mu_eV, double sigma_eV, double *const *gamma_out);
pgb_status pgb_batch_tuning(const pgb_batch *batch, int *tile_q, int *threads, float *cand_ms,
                            int64_t *graph_launches);
pgb_status pgb_batch_set_precision(pgb_batch *batch, int precision);
const char *pgb_batch_last_error(const pgb_batch *batch);
void pgb_batch_destroy(pgb_batch *batch);

/* Replace |g|^2 of every entry of the current list, keeping its rows,
 * columns and modes: g2 [nnz] float32 (host or device), eV^2.  a and b are
 * recomputed as in pgb_build_collision.  For fitting |g|^2 with the
 * derivatives below.                                                         */
pgb_status pgb_collision_set_g2(pgb_ctx *ctx, const float *g2);

/* Reverse-mode derivatives of I[f] (Eq. e_ph_scattering) at f [nstates]:
 * for a covector lam [nstates],
 *   vjp_f[c]  = sum_s lam_s dI_s/df_c            [nstates], 1/s
 *   vjp_g2[e] = sum_s lam_s dI_s/d|g|^2_e        [nnz] in list order, 1/(s eV^2)
 * (vjp_g2 may be NULL).  Any list is accepted: the column sums run over a
 * transposed copy of the list, built on first use and kept with the list.
 * Arithmetic as pgb_collision (FP32 entry products, compensated sums, FP64
 * per state).  All arrays host or device.                                    */
pgb_status pgb_collision_vjp(pgb_ctx *ctx, const double *f, const double *lam, double *vjp_f, double *vjp_g2);

/* Discrete adjoint of pgb_step_rk4 (Sec. 2.1.1 stepping of Eq. e_ph_scattering).
 * Runs nsteps RK4 steps of dt_fs from f0 [nstates] (not modified) exactly as
 * pgb_step_rk4 does, then for a loss L(f(t_end)) with lam_end = dL/df(t_end)
 * [nstates] returns
 *   lam_0  [nstates]  dL/df0 (the reverse-mode derivative of the RK4 steps
 *                     as computed, stage by stage),
 *   dL_dg2 [nnz]      dL/d|g|^2_e in list order, or NULL to skip it,
 *   f_end  [nstates]  f(t_end), bit-identical to pgb_step_rk4, or NULL.
 * f is kept every `checkpoint` steps (values < 1 mean 1); the last segment
 * stores its stage states during the forward pass and every other segment is
 * recomputed once during the reverse sweep (with checkpoint >= nsteps there
 * is no recomputation at all).  Device
 * memory is about (nsteps/checkpoint + 8 checkpoint + 12) nstates doubles,
 * plus 8 nnz bytes with dL_dg2, plus 24 nnz bytes for the transposed list.
 * All arrays host or device.                                                 */
pgb_status pgb_rk4_adjoint(pgb_ctx *ctx, const double *f0, double dt_fs, int64_t nsteps, int64_t checkpoint,
                           const double *lam_end, double *lam_0, double *dL_dg2, double *f_end);

/* Allocation-free scattering rates (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory during the call - a host
 * framework that has already handed the GPU's memory to its own pool, or a
 * service whose request path forbids cudaMalloc because an allocation can
 * synchronise the device.  Computes the same Gamma_nk as
 * pgb_scattering_rates with precision PGB_FP32 (no mode-resolved output), but
 * every temporary lives in one fixed device array of
 * PGB_NOALLOC_SCRATCH_BYTES that the library holds on each GPU until the
 * process exits; the call makes no allocation of any kind.
 *   - k_idx [nk] and gamma_out [nk][nw] must be device pointers on the
 *     context's GPU (no host staging, since that would need a buffer);
 *     otherwise PGB_EINVAL.
 *   - A grid whose scratch for a single k-point exceeds the array returns
 *     PGB_EINVAL with the required size in pgb_last_error(); larger k lists
 *     are processed in batches that fit.
 *   - The first call on each device looks up the array's device address and
 *     keeps it until the process exits: make that first call before any
 *     stream capture, and do not reset the device (cudaDeviceReset) while the
 *     library is loaded.
 *   - Each call checks the k indices on the device and reads the result back,
 *     so it synchronises the context's stream (the host waits for the work
 *     queued before it) before launching the rates kernels.
 *   - All calls share the array and it keeps the last call's contents: calls
 *     that overlap on the GPU race and must be serialised by the caller.    */
#define PGB_NOALLOC_SCRATCH_BYTES (64u << 20)
pgb_status pgb_scattering_rates_noalloc(pgb_ctx *ctx, const int32_t *k_idx, int64_t nk, double T_K,
                                        double mu_eV, double sigma_eV, double *gamma_out);

/* Number of kernel launches this context has issued since creation.         */
int64_t pgb_launch_count(const pgb_ctx *ctx);

/* Kernel timing.  When enabled, the launches of the kernel classes below are
 * bracketed with CUDA events on the context's stream (no synchronisation).
 * pgb_profile_read synchronises the stream, returns the summed device time
 * (ms) and launch count of one class since the last read, and resets them.  */
enum {
    PGB_PROF_QSUM = 0,      /* Fourier sum over R_p for every q (the dominant contraction) */
    PGB_PROF_RSUM = 1,      /* Fourier sum over R_e for every k, with the U(k) fold        */
    PGB_PROF_EPILOGUE = 2,  /* rotation, mode projection, |g|^2, delta weights, Gamma      */
    PGB_PROF_COLLISION = 3, /* collision integral / RK4 stage                              */
    PGB_PROF_BANDS = 4,     /* Fourier sum H(k) = sum_R e^{ik.R} H(R) at off-grid points (FP64, or the
                               double-float cos/sin form of the FP32 paths) */
    PGB_PROF_ADJOINT = 5,   /* transposed-list column pass of the reverse-mode derivatives */
    PGB_PROF_NKERNELS = 6
};
pgb_status pgb_profile(pgb_ctx *ctx, int enable);
pgb_status pgb_profile_read(pgb_ctx *ctx, int kernel_class, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* PERTGB_H */
