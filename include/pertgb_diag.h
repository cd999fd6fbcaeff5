/*
 * pertgb_diag.h - diagnostic entry points of libpertgb (not part of the hot path).
 *
 * They expose intermediate results of the interpolation so that each stage
 * can be checked on its own against a reference.  Conventions as in pertgb.h.
 */
#ifndef PERTGB_DIAG_H
#define PERTGB_DIAG_H

#include "pertgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bands at arbitrary points (Sec. 2.2.1, Eq. wannier_3): for pts [n][3]
 * (host or device) writes H^(W)(k) [n][nw][nw] complex128, eps [n][nw] and
 * U [n][nw][nw] complex128 (columns are eigenvectors).  Any output may be NULL. */
pgb_status pgb_diag_bands(pgb_ctx *ctx, const double *pts, int64_t n, double *Hk, double *eps, double *U);

/* Bands at n points (crystal coordinates [n][3], host or device) by the path the
 * FP32 Monte-Carlo rates use (Sec. 2.2.1, Eq. wannier_3): the packed Hermitian
 * H(k) [n][nw*nw] float64 (nw real diagonal entries, then (re, im) of the
 * entries (i, j), i < j, row by row) from the real cos/sin Fourier sum over one
 * representative of each {R, -R}; eps [n][nw] float64 ascending, refined in
 * FP64; U [n][nw][nw] complex64 (interleaved floats, column n the eigenvector of
 * band n) from the FP32 parallel Jacobi.  Outputs host or device, any may be
 * NULL.  Needs nw >= 2 (PGB_EINVAL otherwise).                               */
pgb_status pgb_diag_bands_mixed(pgb_ctx *ctx, const double *pts, int64_t n, double *Hp, double *eps, float *U);

/* The same for the phonons of the FP32 Monte-Carlo rates (Sec. 2.2.2, Eq. IFC2):
 * Dp [n][nm*nm] the packed mass-scaled D(q) = sum_R e^{iq.R} D(R)/sqrt(M M'),
 * w2 [n][nm] its eigenvalues omega^2 ascending (eV/bohr^2/amu), e [n][nm][nm]
 * complex64 the modes (column nu), refined in FP64 like the eigenvalues.    */
pgb_status pgb_diag_phonons_mixed(pgb_ctx *ctx, const double *pts, int64_t n, double *Dp, double *w2, float *e);

/* The device eigensolver template run on the host for `count` Hermitian
 * n x n complex128 matrices: eval [count][n], evec [count][n][n].
 * Returns 0, or -1 for an unsupported n (supported: 1, 2, 3, 6, 8, 16).     */
int pgb_selftest_heevj(int n, int count, const double *mat, double *eval, double *evec);

/* The device eigensolver kernel on `count` host matrices (as above, n = 1..16). */
pgb_status pgb_selftest_heevj_device(pgb_ctx *ctx, int n, int count, const double *mat, double *eval,
                                     double *evec);

/* Bounded-wait self-test: one GPU thread waits on an mbarrier that nothing
 * arrives on, using the same clock-bounded wait as the tensor-core pipelines
 * (budget in SM clock cycles, 1..2^32).  Returns PGB_ETIMEOUT when the wait
 * ran out and the kernel returned normally, which is the expected result.   */
pgb_status pgb_selftest_wait_timeout(pgb_ctx *ctx, long long budget_cycles);

/* The energy mismatch and Gaussian weight of one term exactly as the fused
 * tensor-core rates epilogue forms them (Sec. 2.1.2, Eqs. scatter_rate,
 * BTE_W): en, em (band energies at k and k+q) and hw (hbar*omega) [n], eV,
 * host or device, are shifted by eps_ref and split into (hi, lo) float pairs
 * like the epilogue's tables; out [n][4] float (host or device) receives
 * x_em = e_n - e_m - hw, x_abs = e_n - e_m + hw and, for |x| <= 7 sigma (else
 * 0), the weights exp(-(x/sigma)^2) of each, all in FP32 as in the kernel.   */
pgb_status pgb_diag_delta_weights(pgb_ctx *ctx, int64_t n, const double *en, const double *em, const double *hw,
                                  double eps_ref, double sigma, float *out);

/* Measured FP64 arithmetic rate of the context's device in TFLOP/s (*tflops):
 * every thread runs sixteen independent chains of dependent FMAs, 2 FLOP each,
 * timed with events (best of three runs after a warm-up).  The denominator of
 * the FP64-bound kernels' rooflines.                                         */
pgb_status pgb_diag_fp64_rate(pgb_ctx *ctx, double *tflops);

/* Device allocations.  Every device allocation the library makes (model and
 * grid tables, scratch, per-call temporaries) goes through one internal call.
 * pgb_diag_alloc_count returns how many it has been asked for since the
 * library was loaded (process-wide, all contexts).  pgb_diag_fail_alloc(n)
 * makes the n-th next one (n = 0: the next) fail on the host with
 * cudaErrorMemoryAllocation, without touching the device, exactly once;
 * n < 0 cancels a pending failure.  The failing entry point returns
 * PGB_ENOMEM and its context stays usable.  Test hook, not thread safe
 * across concurrent callers.                                                */
int64_t pgb_diag_alloc_count(void);
void pgb_diag_fail_alloc(int64_t n);

#ifdef __cplusplus
}
#endif
#endif
