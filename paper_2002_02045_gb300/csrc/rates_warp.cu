// Scattering-rate epilogue for the shapes the fused tensor-core kernel does not
// cover (Sec. 2.2.3 Eqs. eph_mat_wann2 and eph_mat; Sec. 2.1.2 Eqs. scatter_rate
// and BTE_W), fed by the tensor-core q-sum in q slabs that stay in L2.
//
// The q-sum writes C[b][q][n ka i] = sum_p e^{iq.R_p} G_kb[p][n ka i] for one slab
// of q-points (at most 64 MB, so the slab is still in L2 when it is read here).
// One warp per task = (k of the batch, chunk of qc q-points of the slab, band n):
// slabs of wide shapes hold few q-points, so the bands supply the parallelism.
// For each q of the chunk (k+q followed incrementally on the grid) the warp
//   1. screens the (nu, m) of the row 32 at a time against |x| <= 7 sigma (FP32
//      with a margin; e_m(k+q) and hbar*omega_nu(q) held in lanes),
//   2. evaluates each live term as a warp-wide dot product
//        g_mn nu = sum_{ka, i} coef[q][nu][ka] conj(U_im(k+q)) C[q][n][ka][i]
//      (FP32 products: lane = one mode column ka and a block of i, the row of C
//      in registers), four terms at a time,
//   3. queues the terms in lane slots and, 32 at a time, takes their energy
//      differences, Gaussian weights and occupation factors in FP64 with the
//      full warp, then adds them per mode nu in a fixed order (FP32 within a
//      flush, FP64 in the task's accumulators).
// Each task writes its band's entries of one partial block [nu][n];
// launch_rates_reduce adds the blocks of a k in order, so the result does not
// depend on the schedule.
#include <algorithm>

#include "cplx.cuh"
#include "internal.cuh"

namespace pgb {

namespace {

constexpr int kWarps = 8;                       // warps per block
constexpr int kTPL = (kMaxNw * kMaxNmode + 31) / 32;

template <int EL>
__device__ __forceinline__ float2 rot_part(const float2 *__restrict__ u, int stride, const float2 (&cr)[kMaxNw]) {
    float2 rr = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < EL; ++e) cfma_conj(rr, u[e * stride], cr[e]);
    return rr;
}

// sum_i conj(U_im) C[ka][i] over this lane's el elements; U_im at u[e * stride]
__device__ __forceinline__ float2 rot_dispatch(int el, const float2 *__restrict__ u, int stride,
                                               const float2 (&cr)[kMaxNw]) {
    switch (el) {
        case 1: return rot_part<1>(u, stride, cr);
        case 2: return rot_part<2>(u, stride, cr);
        case 3: return rot_part<3>(u, stride, cr);
        case 4: return rot_part<4>(u, stride, cr);
        case 6: return rot_part<6>(u, stride, cr);
        case 8: return rot_part<8>(u, stride, cr);
        default: {
            float2 rr = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < kMaxNw; ++e)
                if (e < el) cfma_conj(rr, u[e * stride], cr[e]);
            return rr;
        }
    }
}

__global__ void __launch_bounds__(32 * kWarps, 2) k_rates_warp(WarpRatesArgs a) {
    __shared__ double acc_s[kWarps][kMaxNmode];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *acc = acc_s[wid];
    const int nw = a.nw, nm = a.nm, P = nm * nw, nc = nm * nw, per = nm * nw;
    const int ib = a.ib, el = nw / ib;
    const bool act = lane < nm * ib;
    const int ka = act ? lane / ib : 0, i0 = act ? (lane - (lane / ib) * ib) * el : 0;
    // screen combos c = 32 j + lane -> (m, nu), m-major so that the live terms of one final
    // band m arrive together and share its rotation; packed as nu * 16 + m, four per word
    uint32_t scm[kTPL / 4] = {0u, 0u};
#pragma unroll
    for (int j = 0; j < kTPL; ++j) {
        const int cc = 32 * j + lane;
        const uint32_t m = cc < nc ? (uint32_t)(cc / nm) : 0u, v = cc < nc ? (uint32_t)(cc - (cc / nm) * nm) : 0u;
        scm[j / 4] |= ((v << 4) | m) << (8 * (j % 4));
    }
    const int nj = (nc + 31) / 32;
    const double is = 1.0 / a.sigma, ycut2 = kDeltaCut * kDeltaCut;
    const float cut32 = (float)(kDeltaCut * a.sigma) + 1e-4f;
    const int kg0 = a.kg[0], kg1 = a.kg[1], kg2 = a.kg[2], qg1 = a.qg[1], qg2 = a.qg[2];
    const int st0 = kg0 / a.qg[0], st1 = kg1 / qg1, st2 = kg2 / qg2;
    const int64_t ntask = a.nb * a.nch * nw;
    for (int64_t task = (int64_t)blockIdx.x * kWarps + wid; task < ntask; task += (int64_t)gridDim.x * kWarps) {
        const int n = (int)(task % nw);
        const int64_t bc = task / nw;
        const int64_t b = bc / a.nch;
        const int ch = (int)(bc - b * a.nch);
        const int64_t ql0 = (int64_t)ch * a.qc;                       // first row of the slab
        const int nq = (int)(a.nqs - ql0 < a.qc ? a.nqs - ql0 : a.qc);
        const int64_t q0 = a.q_off + ql0;                               // its q-grid index
        const int64_t k = a.kidx[b];
        const int k3 = (int)(k % kg2), k2 = (int)((k / kg2) % kg1), k1 = (int)(k / ((int64_t)kg1 * kg2));
        int c3 = (int)(q0 % qg2), c2 = (int)((q0 / qg2) % qg1), c1 = (int)(q0 / ((int64_t)qg1 * qg2));
        for (int r = lane; r < nm; r += 32) acc[r] = 0.0;
        __syncwarp();
        const float en = a.eps32[k * nw + n];
        const double en64 = a.eps[k * nw + n];
        // the term waiting in this lane's slot: |g|^2, nu and the indices of e_m(k+q) and (q, nu)
        int pending = 0, p_key = 0, p_e = 0, p_qv = 0;
        float p_g2 = 0.f;
        auto flush = [&](int count) {
            float contrib = 0.f;
            if (lane < count) {
                const double w = a.hw[p_qv], N = a.nbe[p_qv], f = a.focc[p_e];
                const double d = en64 - a.eps[p_e];
                const double ye = (d - w) * is, ya = (d + w) * is;
                double W = 0.0;
                if (ye * ye <= ycut2) W += exp(-ye * ye) * (1.0 + N - f);
                if (ya * ya <= ycut2) W += exp(-ya * ya) * (N + f);
                contrib = (float)((double)p_g2 * W);
            }
            // per-nu sums of the waiting terms, in order of the lowest lane holding each mode
            unsigned rem = __ballot_sync(0xffffffffu, lane < count);
            while (rem) {
                const int lead = __ffs(rem) - 1;
                const int key = __shfl_sync(0xffffffffu, p_key, lead);
                const unsigned grp = __ballot_sync(0xffffffffu, lane < count && p_key == key);
                rem &= ~grp;
                float sv = ((grp >> lane) & 1u) ? contrib : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                if (lane == 0) acc[key] += (double)sv;
            }
            __syncwarp();
        };
        for (int qq = 0; qq < nq; ++qq) {
            const int64_t q = q0 + qq;
            int t1 = k1 + c1 * st0, t2 = k2 + c2 * st1, t3 = k3 + c3 * st2;
            t1 -= (t1 >= kg0) ? kg0 : 0;
            t2 -= (t2 >= kg1) ? kg1 : 0;
            t3 -= (t3 >= kg2) ? kg2 : 0;
            const int64_t kq = ((int64_t)t1 * kg1 + t2) * kg2 + t3;
            if (++c3 == qg2) {
                c3 = 0;
                if (++c2 == qg1) {
                    c2 = 0;
                    ++c1;
                }
            }
            const float em_l = lane < nw ? a.eps32[kq * nw + lane] : 0.f;
            const float w_l = lane < nm ? a.hw32[q * nm + lane] : 0.f;
            const float2 *Uk = a.U + kq * nw * nw + (int64_t)i0 * nw;   // U[k+q][i][m]: element (i0 + e, m) at + e * nw + m
            const float2 *cq = a.coef + q * nm * nm + ka;
            {
                bool loaded = false;
                int m_rot = -1;   // final band whose rotation rr_m holds (this row)
                float2 rr_m = make_float2(0.f, 0.f);
                float2 cr[kMaxNw];
                for (int j = 0; j < nj; ++j) {
                    const uint32_t vm = (scm[j / 4] >> (8 * (j % 4))) & 0xffu;
                    const float em = __shfl_sync(0xffffffffu, em_l, (int)(vm & 15u));
                    const float w = __shfl_sync(0xffffffffu, w_l, (int)(vm >> 4));
                    bool live = false;
                    if (32 * j + lane < nc && w >= (float)kOmegaMinEv) {
                        const float d = en - em;
                        live = fabsf(d - w) <= cut32 || fabsf(d + w) <= cut32;
                    }
                    unsigned bal = __ballot_sync(0xffffffffu, live);
                    if (bal && !loaded) {
                        const float2 *crow = a.C + (b * a.nqs + ql0 + qq) * a.ldc + (int64_t)n * P + ka * nw + i0;
#pragma unroll
                        for (int e = 0; e < kMaxNw; ++e) cr[e] = (act && e < el) ? crow[e] : make_float2(0.f, 0.f);
                        loaded = true;
                    }
                    while (bal) {
                        constexpr int TB = 4;
                        int cnt = 0;
                        uint32_t tv[TB];
#pragma unroll
                        for (int u = 0; u < TB; ++u) {
                            const int src = bal ? __ffs(bal) - 1 : 0;
                            tv[u] = __shfl_sync(0xffffffffu, vm, src);
                            if (bal) {
                                bal &= bal - 1;
                                ++cnt;
                            }
                        }
                        float2 g[TB];
#pragma unroll
                        for (int u = 0; u < TB; ++u) {
                            g[u] = make_float2(0.f, 0.f);
                            if (u < cnt) {   // warp-uniform
                                const int v = (int)(tv[u] >> 4), m = (int)(tv[u] & 15u);
                                if (m != m_rot) {   // the rotation of final band m, once per run of its terms
                                    rr_m = act ? rot_dispatch(el, Uk + m, nw, cr) : make_float2(0.f, 0.f);
                                    m_rot = m;
                                }
                                if (act) cfma(g[u], cq[v * nm], rr_m);
                            }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                            for (int u = 0; u < TB; ++u) {
                                g[u].x += __shfl_xor_sync(0xffffffffu, g[u].x, o);
                                g[u].y += __shfl_xor_sync(0xffffffffu, g[u].y, o);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < TB; ++u) {
                            if (u >= cnt) break;
                            if (lane == pending) {
                                p_key = (int)(tv[u] >> 4);
                                p_g2 = cabs2(g[u]);
                                p_e = (int)(kq * nw) + (int)(tv[u] & 15u);
                                p_qv = (int)(q * nm) + (int)(tv[u] >> 4);
                            }
                            if (++pending == 32) {
                                flush(32);
                                pending = 0;
                            }
                        }
                    }
                }
            }
        }
        flush(pending);
        double *out = a.partial + ((b * a.nqblk) + a.blk0 + ch) * per + n;
        for (int v = lane; v < nm; v += 32) out[v * nw] = acc[v];
        __syncwarp();
    }
}

}  // namespace

int warp_rates_ib(int nw, int nm) {
    for (int ib : {4, 2})
        if (nm * ib <= 32 && nw % ib == 0) return ib;
    return 1;
}

pgb_status launch_rates_warp(pgb_ctx *c, const WarpRatesArgs &a) {
    const int64_t ntask = a.nb * a.nch * a.nw;
    if (ntask == 0) return PGB_OK;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t grid = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)std::max(sms, 1) * 2);
    k_rates_warp<<<(unsigned)grid, 32 * kWarps, 0, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb
