// Per-entry coefficients of the collision integral (Eq. e_ph_scattering).
#pragma once

#include "internal.cuh"

namespace pgb {

// Geometry and physics shared by every entry of a list.
struct CoeffGeom {
    int nb, band_lo, nw, nm;
    int kg[3];
    const double *eps;   // [Nk][nw]
    const double *hw;    // [Nq][nm] (q grid == k grid)
    double T, sigma, scale;   // scale = (2 pi/hbar) / (N_q sigma sqrt(pi))
};

// geometry of the context's current list (collision.cu)
CoeffGeom coeff_geom(const pgb_ctx *c);

// Gaussian factors and phonon occupation of the entry s -> sp by mode `mode`:
// de = exp(-(x_em/sigma)^2), da = exp(-(x_abs/sigma)^2), x_em = (e_s - e_sp) - hw,
// x_abs = (e_s - e_sp) + hw, N = 1/(e^{hw/kT} - 1).  Returns false (and zeros)
// when hbar*omega < omega_min.
__device__ __forceinline__ bool coll_factors(const CoeffGeom &g, int32_t s, int32_t sp, int32_t mode, double &de,
                                             double &da, double &N) {
    const int64_t k = s / g.nb, kp = sp / g.nb;
    const int n = s % g.nb + g.band_lo, m = sp % g.nb + g.band_lo;
    const int k3 = (int)(k % g.kg[2]), k2 = (int)((k / g.kg[2]) % g.kg[1]), k1 = (int)(k / ((int64_t)g.kg[1] * g.kg[2]));
    const int l3 = (int)(kp % g.kg[2]), l2 = (int)((kp / g.kg[2]) % g.kg[1]),
              l1 = (int)(kp / ((int64_t)g.kg[1] * g.kg[2]));
    const int q1 = (l1 - k1 + g.kg[0]) % g.kg[0], q2 = (l2 - k2 + g.kg[1]) % g.kg[1], q3 = (l3 - k3 + g.kg[2]) % g.kg[2];
    // q and -q have the same frequencies; the smaller of the two indices is
    // used so that both directions of a process see bit-identical hw
    const int64_t q = ((int64_t)q1 * g.kg[1] + q2) * g.kg[2] + q3;
    const int r1 = (g.kg[0] - q1) % g.kg[0], r2 = (g.kg[1] - q2) % g.kg[1], r3 = (g.kg[2] - q3) % g.kg[2];
    const int64_t qm = ((int64_t)r1 * g.kg[1] + r2) * g.kg[2] + r3;
    const double w = g.hw[(q < qm ? q : qm) * g.nm + mode];
    de = 0.0;
    da = 0.0;
    N = 0.0;
    if (!(w >= kOmegaMinEv)) return false;
    N = 1.0 / expm1(w / (kBoltzEvK * g.T));
    const double d = g.eps[k * g.nw + n] - g.eps[kp * g.nw + m];
    const double is = 1.0 / g.sigma;
    const double xe = __dmul_rn(__dsub_rn(d, w), is), xa = __dmul_rn(__dadd_rn(d, w), is);
    de = exp(-__dmul_rn(xe, xe));
    da = exp(-__dmul_rn(xa, xa));
    return true;
}

// Emission / absorption brackets of the entry s -> sp by mode `mode`, per unit |g|^2,
// without the scale:  ca = d_em (N+1) + d_abs N,  cb = d_em N + d_abs (N+1).
// The reverse entry sp -> s sees the exact negation of e_s - e_sp, so its x_em is
// -x_abs of this entry: the products are rounded separately (no contraction) and
// the sums commute, so ca of the reverse entry equals cb of this one bit for bit.
// Both are 0 when hbar*omega < omega_min.
__device__ __forceinline__ void coll_brackets(const CoeffGeom &g, int32_t s, int32_t sp, int32_t mode, double &ca,
                                              double &cb) {
    double de, da, N;
    ca = 0.0;
    cb = 0.0;
    if (!coll_factors(g, s, sp, mode, de, da, N)) return;
    const double N1 = __dadd_rn(N, 1.0);
    ca = __dadd_rn(__dmul_rn(de, N1), __dmul_rn(da, N));
    cb = __dadd_rn(__dmul_rn(de, N), __dmul_rn(da, N1));
}

}  // namespace pgb
