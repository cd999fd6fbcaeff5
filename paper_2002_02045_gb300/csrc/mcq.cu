// Monte-Carlo q sampling of the scattering rates (Sec. 4.3, random q uniform or
// Cauchy) and the carrier population by the linear tetrahedron method (Eq. pop).
//
// Rates at arbitrary k with random q: the caller's uniforms u in [0,1)^3 map to
//   uniform: q_i = u_i - 1/2, p(q) = 1;
//   Cauchy:  q_i = atan(c tan(pi (u_i - 1/2))) / pi, p(q_i) = c / (c^2 cos^2(pi q_i) + sin^2(pi q_i)),
// and Gamma_nk = (1/N) sum_j y_j with y_j = sum_{m nu} W(q_j) / p(q_j).  k + q is off the
// grid, so bands at every (k, q_j) are diagonalised; the per-pair epilogue reads
// U(k+q) and e(k+q) from those arrays.  Per (k, n) the sums of y and y^2 give the
// estimate and its standard error; partial sums per block are added in a
// fixed order (deterministic).
//
// Population: N(E) = sum_n (1/V_BZ) int f_n(k) theta(E - e_n(k)) dk with e and f
// linear on each of the six tetrahedra of every grid cell (corner weights of
// the linear tetrahedron method); one block per energy, threads over
// (tetrahedron, band), fixed-order block reduction.
#include <cmath>

#include "cplx.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

__global__ void k_mc_qpoints(int64_t nq, const double *__restrict__ u, int sampling, double c,
                             double *__restrict__ q, double *__restrict__ pinv) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq) return;
    double w = 1.0;
    for (int i = 0; i < 3; ++i) {
        const double x = u[3 * t + i] - 0.5;
        if (sampling == PGB_Q_CAUCHY) {
            const double qi = atan(c * tan(kPi * x)) / kPi;
            const double cs = cos(kPi * qi), sn = sin(kPi * qi);
            w *= (c * c * cs * cs + sn * sn) / c;   // 1 / p(q_i)
            q[3 * t + i] = qi;
        } else {
            q[3 * t + i] = x;
        }
    }
    pinv[t] = w;
}

struct McArgs {
    int64_t nkb, nq;            // k-points of this batch, q samples of this chunk
    int nw, nm;
    const void *C;              // [nkb][nq][ldc], columns (n, ka, i) first
    int64_t ldc;
    const void *Ukq;            // [nkb*nq][nw][nw]
    const double *eps_k;        // [nkb][nw]
    const double *eps_kq;       // [nkb*nq][nw]
    const double *hw;           // [nq][nm]
    const void *coef;           // [nq][nm][nm]
    const double *pinv;         // [nq]
    double T, mu, sigma;
    int qpb;                    // q per block
    double *partial;            // [nkb][nblk][nw][2]
};

template <typename T>
__global__ void __launch_bounds__(256) k_mc_epilogue(McArgs a) {
    using T2 = V2<T>;
    extern __shared__ double red[];                 // [qpb][nw][2], then f [qpb][nw], then N [qpb][nm]
    const int nw = a.nw, nm = a.nm;
    const int ql = threadIdx.x / nw;
    const int n = threadIdx.x % nw;
    const int64_t b = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x * a.qpb + ql;
    const double kT = kBoltzEvK * a.T;
    // occupations f(e_m(k+q)) and Bose factors N(omega_nu(q)) of the block's q-points,
    // once each (every thread of a q-point uses them)
    double *sf = red + 2 * a.qpb * nw, *sN = sf + a.qpb * nw;
    for (int x = threadIdx.x; x < a.qpb * nw; x += blockDim.x) {
        const int64_t qq = (int64_t)blockIdx.x * a.qpb + x / nw;
        sf[x] = qq < a.nq ? 1.0 / (exp((a.eps_kq[(b * a.nq + qq) * nw + x % nw] - a.mu) / kT) + 1.0) : 0.0;
    }
    for (int x = threadIdx.x; x < a.qpb * nm; x += blockDim.x) {
        const int64_t qq = (int64_t)blockIdx.x * a.qpb + x / nm;
        const double w = qq < a.nq ? a.hw[qq * nm + x % nm] : 0.0;
        sN[x] = w >= kOmegaMinEv ? 1.0 / expm1(w / kT) : 0.0;
    }
    __syncthreads();
    double y = 0.0;
    if (ql < a.qpb && q < a.nq) {
        const int64_t pr = b * a.nq + q;            // pair index
        const double en = a.eps_k[b * nw + n];
        const double is = 1.0 / a.sigma, ycut2 = kDeltaCut * kDeltaCut;
        const T2 *Cn = (const T2 *)a.C + pr * a.ldc + (int64_t)n * nm * nw;
        const T2 *U = (const T2 *)a.Ukq + pr * nw * nw;
        const double *em = a.eps_kq + pr * nw;
        double acc = 0.0;
        // FP32 copies for the screen: |x| <= 7 sigma with a margin of 1e-4 eV (FP32
        // rounding of energies of a few eV is ~1e-6 eV); survivors take the exact FP64 test
        float em32[kMaxNw];
#pragma unroll
        for (int m = 0; m < kMaxNw; ++m) em32[m] = m < nw ? (float)em[m] : 0.f;
        const float en32 = (float)en, cut32 = (float)(kDeltaCut * a.sigma) + 1e-4f;
        for (int v = 0; v < nm; ++v) {
            const double w = a.hw[q * nm + v];
            if (!(w >= kOmegaMinEv)) continue;
            const float w32 = (float)w;
            // screen before the projection
            uint32_t live = 0;
#pragma unroll
            for (int m = 0; m < kMaxNw; ++m) {
                if (m >= nw) break;
                const float d = en32 - em32[m];
                if (fabsf(d - w32) <= cut32 || fabsf(d + w32) <= cut32) live |= 1u << m;
            }
            if (!live) continue;
            const T2 *cf = (const T2 *)a.coef + (q * nm + v) * nm;
            T2 gv[kMaxNw];
#pragma unroll
            for (int i = 0; i < kMaxNw; ++i) gv[i] = cmake<T>(0, 0);
            for (int ka = 0; ka < nm; ++ka) {
                const T2 cc = cf[ka];
#pragma unroll
                for (int i = 0; i < kMaxNw; ++i)
                    if (i < nw) cfma(gv[i], cc, Cn[ka * nw + i]);
            }
            const double N = sN[ql * nm + v];
            while (live) {
                const int m = __ffs(live) - 1;
                live &= live - 1;
                T2 g = cmake<T>(0, 0);
#pragma unroll
                for (int i = 0; i < kMaxNw; ++i)
                    if (i < nw) cfma_conj(g, U[i * nw + m], gv[i]);
                const double g2 = (double)cabs2(g);
                const double d = en - em[m];
                const double ye = (d - w) * is, ya = (d + w) * is;
                const double fm = sf[ql * nw + m];
                double W = 0.0;
                if (ye * ye <= ycut2) W += exp(-ye * ye) * (1.0 + N - fm);
                if (ya * ya <= ycut2) W += exp(-ya * ya) * (N + fm);
                acc += g2 * W;
            }
        }
        y = acc * a.pinv[q];
    }
    red[(ql * nw + n) * 2] = y;
    red[(ql * nw + n) * 2 + 1] = y * y;
    __syncthreads();
    for (int r = threadIdx.x; r < 2 * nw; r += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < a.qpb; ++l) s += red[l * 2 * nw + r];
        a.partial[(b * gridDim.x + blockIdx.x) * 2 * nw + r] = s;
    }
}

// acc[k][n][2] += sum over the blocks of this chunk, in block order
__global__ void k_mc_accum(int64_t nkb, int nblk, int nw, const double *__restrict__ partial,
                           double *__restrict__ acc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nkb * 2 * nw) return;
    const int64_t b = t / (2 * nw);
    const int r = (int)(t % (2 * nw));
    double s = 0.0;
    for (int i = 0; i < nblk; ++i) s += partial[(b * nblk + i) * 2 * nw + r];
    acc[t] += s;
}

__global__ void k_mc_finish(int64_t n, int64_t nq, double scale, const double *__restrict__ acc,
                            double *__restrict__ gamma, double *__restrict__ err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double s1 = acc[2 * t], s2 = acc[2 * t + 1];
    const double mean = s1 / (double)nq;
    gamma[t] = scale * mean;
    if (err) {
        const double var = nq > 1 ? fmax(0.0, (s2 - s1 * mean) / (double)(nq - 1)) : 0.0;
        err[t] = scale * sqrt(var / (double)nq);
    }
}

// ---------------------------------------------------------------------------
// tetrahedron population
// ---------------------------------------------------------------------------
// Corner weights of int_T f theta(E - e) dV / V_T for e, f linear on T, for the
// corner energies in ascending order (s[0] <= ... <= s[3]).
__device__ void tetra_weights_sorted(const double s[4], double E, double w[4]) {
    const double e1 = s[0], e2 = s[1], e3 = s[2], e4 = s[3];
    w[0] = w[1] = w[2] = w[3] = 0.0;
    if (E < e1) return;
    if (E >= e4) {
        w[0] = w[1] = w[2] = w[3] = 0.25;
        return;
    }
    if (E < e2) {
        const double d1 = E - e1, d21 = e2 - e1, d31 = e3 - e1, d41 = e4 - e1;
        const double C = 0.25 * d1 * d1 * d1 / (d21 * d31 * d41);
        w[0] = C * (4.0 - d1 * (1.0 / d21 + 1.0 / d31 + 1.0 / d41));
        w[1] = C * d1 / d21;
        w[2] = C * d1 / d31;
        w[3] = C * d1 / d41;
    } else if (E < e3) {
        const double a1 = E - e1, a2 = E - e2, b3 = e3 - E, b4 = e4 - E;
        const double d31 = e3 - e1, d41 = e4 - e1, d32 = e3 - e2, d42 = e4 - e2;
        const double C1 = 0.25 * a1 * a1 / (d41 * d31);
        const double C2 = 0.25 * a1 * a2 * b3 / (d41 * d32 * d31);
        const double C3 = 0.25 * a2 * a2 * b4 / (d42 * d32 * d41);
        w[0] = C1 + (C1 + C2) * b3 / d31 + (C1 + C2 + C3) * b4 / d41;
        w[1] = C1 + C2 + C3 + (C2 + C3) * b3 / d32 + C3 * b4 / d42;
        w[2] = (C1 + C2) * a1 / d31 + (C2 + C3) * a2 / d32;
        w[3] = (C1 + C2 + C3) * a1 / d41 + C3 * a2 / d42;
    } else {
        const double b4 = e4 - E, d41 = e4 - e1, d42 = e4 - e2, d43 = e4 - e3;
        const double C = 0.25 * b4 * b4 * b4 / (d41 * d42 * d43);
        w[0] = 0.25 - C * b4 / d41;
        w[1] = 0.25 - C * b4 / d42;
        w[2] = 0.25 - C * b4 / d43;
        w[3] = 0.25 - C * (4.0 - b4 * (1.0 / d41 + 1.0 / d42 + 1.0 / d43));
    }
}

constexpr int kPopThreads = 256;

__global__ void __launch_bounds__(kPopThreads) k_population(int n1, int n2, int n3, int nb,
                                                            const double *__restrict__ eps_state,
                                                            const double *__restrict__ f,
                                                            const double *__restrict__ E, double *__restrict__ out) {
    __shared__ double red[kPopThreads / 32];
    const double Ej = E[blockIdx.x];
    const int64_t ncell = (int64_t)n1 * n2 * n3;
    const int64_t total = 6 * ncell * nb;
    // corners of the cube (bits: x, y, z) along the six paths from 0 to 7
    const int path[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < total; t += kPopThreads) {
        const int n = (int)(t % nb);
        const int64_t tc = t / nb;
        const int64_t cell = tc % ncell;
        const int p = (int)(tc / ncell);
        const int i3 = (int)(cell % n3), i2 = (int)((cell / n3) % n2), i1 = (int)(cell / ((int64_t)n2 * n3));
        double e[4], fv[4];
        for (int v = 0; v < 4; ++v) {
            const int cidx = path[p][v];
            // corner bits: 1 = first axis, 2 = second axis, 4 = third axis
            int j1 = i1 + (cidx & 1), j2 = i2 + ((cidx >> 1) & 1), j3 = i3 + ((cidx >> 2) & 1);
            if (j1 == n1) j1 = 0;
            if (j2 == n2) j2 = 0;
            if (j3 == n3) j3 = 0;
            const int64_t s = (((int64_t)j1 * n2 + j2) * n3 + j3) * nb + n;
            e[v] = eps_state[s];
            fv[v] = f[s];
        }
        // sort corners by energy (stable), carrying f
        for (int i = 1; i < 4; ++i)
            for (int j = i; j > 0 && e[j] < e[j - 1]; --j) {
                double x = e[j];
                e[j] = e[j - 1];
                e[j - 1] = x;
                x = fv[j];
                fv[j] = fv[j - 1];
                fv[j - 1] = x;
            }
        double w[4];
        tetra_weights_sorted(e, Ej, w);
        acc += w[0] * fv[0] + w[1] * fv[1] + w[2] * fv[2] + w[3] * fv[3];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kPopThreads / 32; ++w) s += red[w];
        out[blockIdx.x] = s / (double)(6 * ncell);
    }
}

}  // namespace

pgb_status launch_mc_qpoints(pgb_ctx *c, int64_t nq, const double *u, int sampling, double width, double *q,
                             double *pinv) {
    if (nq == 0) return PGB_OK;
    k_mc_qpoints<<<div_up(nq, 256), 256, 0, c->stream>>>(nq, u, sampling, width, q, pinv);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_mc_epilogue(pgb_ctx *c, bool fp32, int64_t nkb, int64_t nq, const void *C, int64_t ldc,
                              const void *Ukq, const double *eps_k, const double *eps_kq, const double *hw,
                              const void *coef, const double *pinv, double T, double mu, double sigma, double *partial,
                              double *acc) {
    if (nkb == 0 || nq == 0) return PGB_OK;
    McArgs a;
    a.nkb = nkb;
    a.nq = nq;
    a.nw = c->nw;
    a.nm = c->nm;
    a.C = C;
    a.ldc = ldc;
    a.Ukq = Ukq;
    a.eps_k = eps_k;
    a.eps_kq = eps_kq;
    a.hw = hw;
    a.coef = coef;
    a.pinv = pinv;
    a.T = T;
    a.mu = mu;
    a.sigma = sigma;
    a.qpb = 256 / c->nw;
    a.partial = partial;
    const int nblk = (int)((nq + a.qpb - 1) / a.qpb);
    dim3 grid((unsigned)nblk, (unsigned)nkb);
    const size_t sh = (size_t)a.qpb * (3 * c->nw + c->nm) * sizeof(double);
    if (fp32)
        k_mc_epilogue<float><<<grid, a.qpb * c->nw, sh, c->stream>>>(a);
    else
        k_mc_epilogue<double><<<grid, a.qpb * c->nw, sh, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    k_mc_accum<<<div_up(nkb * 2 * c->nw, 256), 256, 0, c->stream>>>(nkb, nblk, c->nw, partial, acc);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

int64_t mc_partial_count(const pgb_ctx *c, int64_t nkb, int64_t nq) {
    const int qpb = 256 / c->nw;
    return nkb * ((nq + qpb - 1) / qpb) * 2 * c->nw;
}

pgb_status launch_mc_finish(pgb_ctx *c, int64_t nk, int64_t nq, double sigma, const double *acc, double *gamma,
                            double *err) {
    const int64_t n = nk * c->nw;
    if (n == 0) return PGB_OK;
    const double scale = kTwoPiOverHbar / (sigma * kSqrtPi);
    k_mc_finish<<<div_up(n, 256), 256, 0, c->stream>>>(n, nq, scale, acc, gamma, err);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status launch_population(pgb_ctx *c, const double *f, const double *E, int64_t nE, double *out) {
    if (nE == 0) return PGB_OK;
    const int nb = c->band_hi - c->band_lo;
    k_population<<<(unsigned)nE, kPopThreads, 0, c->stream>>>(c->kg[0], c->kg[1], c->kg[2], nb, c->d_eps_state, f,
                                                             E, out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb
