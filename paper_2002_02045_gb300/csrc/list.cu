// Scattering list on the k grid (Sec. 4.3: (k,q) pairs whose initial and final
// states both lie in the energy window, k+q on the k grid) with |g|^2 from the
// interpolation (Eqs. eph_mat_wann2, eph_mat).
//
// Each unordered process {s, s'} by mode nu is evaluated once, in the
// direction s <= s' (initial band at k, final band at k+q), and written to
// both rows with the same |g|^2: the hermiticity of the perturbation gives the
// reverse process (s' -> s at -q) the same |g|^2, and sharing the value makes
// the sum of I[f] over states vanish to rounding.  A term is kept when one of
// its Gaussian factors has |x| <= 7 sigma (the rates screen).
//
//   count kernel: number of kept entries (no interpolation needed);
//   fill kernel:  per (k, k' in the window, band n), q = k' - k, the mode
//                 projection and rotation of the kept terms, appended with
//                 warp-aggregated atomics as
//                 (key = (s * ns + s') * nmode + nu, |g|^2);
//   a radix sort of the keys gives the deterministic row-major order, and a
//   decode kernel splits the keys into row, col, mode.
#include <cub/device/device_radix_sort.cuh>

#include "cplx.cuh"
#include "internal.cuh"

namespace pgb {

namespace {
inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

// q index of k' - k on the grid (k grid = q grid)
__device__ __forceinline__ int kdiff_grid(int kp, int k, int n0, int n1, int n2) {
    const int k3 = k % n2, k2 = (k / n2) % n1, k1 = k / (n1 * n2);
    const int l3 = kp % n2, l2 = (kp / n2) % n1, l1 = kp / (n1 * n2);
    return (((l1 - k1 + n0) % n0) * n1 + (l2 - k2 + n1) % n1) * n2 + (l3 - k3 + n2) % n2;
}

__device__ __forceinline__ int kplusq_grid(int k, int q, int n0, int n1, int n2) {
    const int k3 = k % n2, k2 = (k / n2) % n1, k1 = k / (n1 * n2);
    const int q3 = q % n2, q2 = (q / n2) % n1, q1 = q / (n1 * n2);
    int t1 = k1 + q1, t2 = k2 + q2, t3 = k3 + q3;
    t1 -= (t1 >= n0) ? n0 : 0;
    t2 -= (t2 >= n1) ? n1 : 0;
    t3 -= (t3 >= n2) ? n2 : 0;
    return (t1 * n1 + t2) * n2 + t3;
}

struct ListArgs {
    int nb;                  // k-points of this batch
    const int32_t *kidx;     // [nb] k-grid indices
    int Nk;                  // k grid = q grid
    int n0, n1, n2;
    int nw, nm, band_lo, nbnd;
    const int32_t *win;      // [na] k-points with a window state (the only k' = k + q kept)
    int na;
    const float2 *C;         // [nb][na][nbnd][nm][nw]  Rp-summed g with U(k) folded, q = win[w] - k
    const float2 *U;         // [Nk][i][m] FP32
    const float2 *coef;      // [Nq][nu][ka] FP32
    const double *eps;       // [Nk][nw]
    const double *hw;        // [Nq][nm]
    const uint8_t *inwin;    // [Nk * nbnd]
    double cut;              // 7 sigma
    unsigned long long *counter;
    uint64_t *keys;
    float *vals;
    unsigned long long cap;
};

// Whether the term s -> s' by mode nu is one of the kept, canonical entries.
__device__ __forceinline__ bool entry_kept(const ListArgs &a, int s, int sp, double es, double esp, double w) {
    if (s > sp || !a.inwin[sp] || w < kOmegaMinEv) return false;
    const double d = es - esp;
    return fabs(d - w) <= a.cut || fabs(d + w) <= a.cut;
}

// Entries written per kept term: both directions, once if s == s'.
__global__ void k_list_count(ListArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (t < (int64_t)a.nb * a.na) {
        const int b = (int)(t / a.na), w = (int)(t % a.na);
        const int k = a.kidx[b];
        const int kq = a.win[w];
        const int q = kdiff_grid(kq, k, a.n0, a.n1, a.n2);
        for (int nl = 0; nl < a.nbnd; ++nl) {
            const int s = k * a.nbnd + nl;
            if (!a.inwin[s]) continue;
            const double es = a.eps[(int64_t)k * a.nw + a.band_lo + nl];
            for (int ml = 0; ml < a.nbnd; ++ml) {
                const int sp = kq * a.nbnd + ml;
                const double esp = a.eps[(int64_t)kq * a.nw + a.band_lo + ml];
                for (int v = 0; v < a.nm; ++v)
                    if (entry_kept(a, s, sp, es, esp, a.hw[(int64_t)q * a.nm + v])) cnt += (s == sp) ? 1 : 2;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.counter, cnt);
}

// One thread per (b, w, nl).  First pass counts its entries, a warp scan and
// one atomic reserve the slots, second pass computes |g|^2 and writes.
__global__ void k_list_fill(ListArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)a.nb * a.na * a.nbnd;
    int b = 0, q = 0, w = 0, nl = 0, k = 0, kq = 0, s = 0;
    double es = 0.0;
    unsigned cnt = 0;
    const bool act = t < total;
    if (act) {
        nl = (int)(t % a.nbnd);
        w = (int)((t / a.nbnd) % a.na);
        b = (int)(t / ((int64_t)a.nbnd * a.na));
        k = a.kidx[b];
        kq = a.win[w];
        q = kdiff_grid(kq, k, a.n0, a.n1, a.n2);
        s = k * a.nbnd + nl;
        if (a.inwin[s]) {
            es = a.eps[(int64_t)k * a.nw + a.band_lo + nl];
            for (int ml = 0; ml < a.nbnd; ++ml) {
                const int sp = kq * a.nbnd + ml;
                const double esp = a.eps[(int64_t)kq * a.nw + a.band_lo + ml];
                for (int v = 0; v < a.nm; ++v)
                    if (entry_kept(a, s, sp, es, esp, a.hw[(int64_t)q * a.nm + v])) cnt += (s == sp) ? 1 : 2;
            }
        }
    }
    // warp-aggregated reservation
    unsigned incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned wtot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && wtot) base = atomicAdd(a.counter, (unsigned long long)wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned long long pos = base + (incl - cnt);
    if (!act || cnt == 0) return;

    const int ns = a.Nk * a.nbnd;
    const int per_n = a.nm * a.nw;
    const float2 *Cn = a.C + (((int64_t)b * a.na + w) * a.nbnd + nl) * per_n;
    const float2 *cf = a.coef + (int64_t)q * a.nm * a.nm;
    const float2 *U = a.U + (int64_t)kq * a.nw * a.nw;
    for (int v = 0; v < a.nm; ++v) {
        const double hw = a.hw[(int64_t)q * a.nm + v];
        bool anym = false;
        for (int ml = 0; ml < a.nbnd; ++ml) {
            const int sp = kq * a.nbnd + ml;
            anym |= entry_kept(a, s, sp, es, a.eps[(int64_t)kq * a.nw + a.band_lo + ml], hw);
        }
        if (!anym) continue;
        float2 gv[kMaxNw];
#pragma unroll
        for (int i = 0; i < kMaxNw; ++i) gv[i] = make_float2(0.f, 0.f);
        for (int ka = 0; ka < a.nm; ++ka) {
            const float2 c = cf[v * a.nm + ka];
#pragma unroll
            for (int i = 0; i < kMaxNw; ++i)
                if (i < a.nw) cfma(gv[i], c, Cn[ka * a.nw + i]);
        }
        for (int ml = 0; ml < a.nbnd; ++ml) {
            const int sp = kq * a.nbnd + ml;
            if (!entry_kept(a, s, sp, es, a.eps[(int64_t)kq * a.nw + a.band_lo + ml], hw)) continue;
            const int m = a.band_lo + ml;
            float2 g = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < kMaxNw; ++i)
                if (i < a.nw) cfma_conj(g, U[i * a.nw + m], gv[i]);
            const float g2 = g.x * g.x + g.y * g.y;
            if (pos < a.cap) {
                a.keys[pos] = ((uint64_t)s * ns + sp) * a.nm + v;
                a.vals[pos] = g2;
            }
            ++pos;
            if (sp != s) {
                if (pos < a.cap) {
                    a.keys[pos] = ((uint64_t)sp * ns + s) * a.nm + v;
                    a.vals[pos] = g2;
                }
                ++pos;
            }
        }
    }
}

// A operand of the restricted q-sum: row w of batch b is the q-table row of
// q = win[w] - kidx[b]
__global__ void k_gather_qrows(int nb, const int32_t *__restrict__ kidx, int na, const int32_t *__restrict__ win,
                               int n0, int n1, int n2, int nK, const float2 *__restrict__ phq, float2 *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb * na * nK) return;
    const int p = (int)(t % nK);
    const int64_t bw = t / nK;
    const int w = (int)(bw % na), b = (int)(bw / na);
    const int q = kdiff_grid(win[w], kidx[b], n0, n1, n2);
    out[t] = phq[(int64_t)q * nK + p];
}

__global__ void k_list_decode(int64_t n, int ns, int nm, const uint64_t *__restrict__ keys,
                              const float *__restrict__ vals, int32_t *__restrict__ row, int32_t *__restrict__ col,
                              int32_t *__restrict__ mode, float *__restrict__ g2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint64_t key = keys[t];
    mode[t] = (int32_t)(key % nm);
    const uint64_t pair = key / nm;
    col[t] = (int32_t)(pair % ns);
    row[t] = (int32_t)(pair / ns);
    g2[t] = vals[t];
}

}  // namespace

pgb_status list_count(pgb_ctx *c, const ListLaunch &L, unsigned long long *d_counter) {
    ListArgs a;
    a.nb = (int)L.nb;
    a.kidx = L.kidx;
    a.Nk = (int)c->Nk;
    a.n0 = c->kg[0];
    a.n1 = c->kg[1];
    a.n2 = c->kg[2];
    a.nw = c->nw;
    a.nm = c->nm;
    a.band_lo = L.band_lo;
    a.nbnd = L.nbnd;
    a.win = L.win;
    a.na = (int)L.na;
    a.C = nullptr;
    a.U = c->d_U32;
    a.coef = c->d_coef32;
    a.eps = c->d_eps;
    a.hw = c->d_hw;
    a.inwin = L.inwin;
    a.cut = L.cut;
    a.counter = d_counter;
    a.keys = nullptr;
    a.vals = nullptr;
    a.cap = 0;
    const int64_t n = L.nb * L.na;
    if (n == 0) return PGB_OK;
    k_list_count<<<div_up(n, 256), 256, 0, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status list_fill(pgb_ctx *c, const ListLaunch &L, const void *C, unsigned long long *d_counter, uint64_t *keys,
                     float *vals, unsigned long long cap) {
    ListArgs a;
    a.nb = (int)L.nb;
    a.kidx = L.kidx;
    a.Nk = (int)c->Nk;
    a.n0 = c->kg[0];
    a.n1 = c->kg[1];
    a.n2 = c->kg[2];
    a.nw = c->nw;
    a.nm = c->nm;
    a.band_lo = L.band_lo;
    a.nbnd = L.nbnd;
    a.win = L.win;
    a.na = (int)L.na;
    a.C = (const float2 *)C;
    a.U = c->d_U32;
    a.coef = c->d_coef32;
    a.eps = c->d_eps;
    a.hw = c->d_hw;
    a.inwin = L.inwin;
    a.cut = L.cut;
    a.counter = d_counter;
    a.keys = keys;
    a.vals = vals;
    a.cap = cap;
    const int64_t n = L.nb * L.na * L.nbnd;
    if (n == 0) return PGB_OK;
    k_list_fill<<<div_up(n, 256), 256, 0, c->stream>>>(a);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

pgb_status list_sort_decode(pgb_ctx *c, int64_t n, int ns, uint64_t *keys, float *vals, uint64_t *keys_alt,
                            float *vals_alt, int32_t *row, int32_t *col, int32_t *mode, float *g2) {
    if (n == 0) return PGB_OK;
    int end_bit = 1;
    const unsigned long long maxkey = (unsigned long long)ns * ns * c->nm;
    while (end_bit < 64 && (1ull << end_bit) < maxkey) ++end_bit;
    cub::DoubleBuffer<uint64_t> dk(keys, keys_alt);
    cub::DoubleBuffer<float> dv(vals, vals_alt);
    size_t tmp_bytes = 0;
    PGB_CUDA_TRY(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, dk, dv, n, 0, end_bit, c->stream));
    void *tmp = nullptr;
    PGB_CUDA_TRY(c, dev_malloc_async(&tmp, tmp_bytes, c->stream));
    cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, dk, dv, n, 0, end_bit, c->stream);
    cudaFreeAsync(tmp, c->stream);
    PGB_CUDA_TRY(c, e);
    c->launches += 1;
    k_list_decode<<<div_up(n, 256), 256, 0, c->stream>>>(n, ns, c->nm, dk.Current(), dv.Current(), row, col, mode,
                                                          g2);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}

}  // namespace pgb

namespace pgb {
pgb_status list_gather_qrows(pgb_ctx *c, const ListLaunch &L, const void *phq, void *out) {
    const int64_t n = L.nb * L.na * (int64_t)c->nKp;
    if (n == 0) return PGB_OK;
    k_gather_qrows<<<div_up(n, 256), 256, 0, c->stream>>>((int)L.nb, L.kidx, (int)L.na, L.win, c->kg[0], c->kg[1],
                                                          c->kg[2], c->nKp, (const float2 *)phq, (float2 *)out);
    PGB_LAUNCH_CHECK(c);
    return PGB_OK;
}
}  // namespace pgb
