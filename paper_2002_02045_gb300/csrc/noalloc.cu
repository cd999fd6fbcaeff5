// Scattering rates without any device allocation in the call.
//
// Some callers cannot allocate device memory while they run: a host framework
// that has already given all of the GPU's memory to its own pool, or a
// service that forbids cudaMalloc on its request path because an allocation
// can synchronise the whole device and stall other work.  This entry point
// runs the FP32 scattering-rate path with every temporary (phase table,
// Fourier partial sums, occupation tables, per-block partials) carved out of
// one fixed, file-scope device array, so the call itself allocates nothing.
// It exists for those callers only; it has no counterpart in the paper.
//
// Every GPU that loads the library keeps this array until the process exits.
// All calls share it and it keeps the previous call's contents, so calls
// that overlap on the GPU (different streams or contexts on one device) race
// on it and must be serialised by the caller.  The first call on each device
// looks up the array's device address and keeps it for the life of the
// process (so the device must not be reset with cudaDeviceReset while the
// library is loaded); make that first call before any stream capture.  Every
// call reads its k-index check back to the host, so it synchronises the
// context's stream before it launches the rates kernels.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace pgb {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PGB_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the array's host-side name is not a device address).
pgb_status scratch_address(pgb_ctx *c, unsigned char **out) {
    if (c->device < 0 || c->device >= kMaxDevices) {
        c->err = "scattering_rates_noalloc: device index out of range";
        return PGB_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[c->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            c->err = std::string("scattering_rates_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return PGB_ECUDA;
        }
        g_scratch_ptr[c->device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[c->device]);
    return PGB_OK;
}

// Device (or managed) memory of the context's own GPU: a buffer on another GPU
// would be read and written from this one.
bool on_device(const void *p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_check_kidx(const int32_t *__restrict__ kidx, int64_t nk, int64_t Nk, int *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nk && (kidx[t] < 0 || kidx[t] >= Nk)) atomicOr(bad, 1);
}

}  // namespace
}  // namespace pgb

using namespace pgb;

extern "C" pgb_status pgb_scattering_rates_noalloc(pgb_ctx *c, const int32_t *k_idx, int64_t nk, double T,
                                                   double mu, double sigma, double *gamma_out) {
    if (!c) return PGB_EINVAL;
    cudaSetDevice(c->device);
    if (!c->has_grids) {
        c->err = "scattering_rates_noalloc: call set_grids first";
        return PGB_ESTATE;
    }
    if (nk < 0 || !(T > 0.0) || !(sigma > 0.0) || !std::isfinite(mu)) {
        c->err = "scattering_rates_noalloc: need nk >= 0, T > 0, sigma > 0, finite mu";
        return PGB_EINVAL;
    }
    if (nk == 0) return PGB_OK;
    if (!k_idx || !gamma_out || !on_device(k_idx, c->device) || !on_device(gamma_out, c->device)) {
        c->err = "scattering_rates_noalloc: k_idx and gamma_out must be device pointers on the context's GPU";
        return PGB_EINVAL;
    }
    const int nw = c->nw, nm = c->nm;
    const int64_t ncol = (int64_t)nm * nw * nw, nrow = (int64_t)c->nKp * ncol, nrowS = (int64_t)c->nRgp * ncol;
    const size_t es = sizeof(float2);
    const int per = nm * nw;
    const int qpb = std::max(1, 256 / nw);
    const int qiters = 8;
    const int64_t nqblk = (c->Nq + (int64_t)qpb * qiters - 1) / ((int64_t)qpb * qiters);

    // fixed part: q phase table and occupation tables; per-k part: Fourier sums and partials
    const size_t fixed = 256 + al256((size_t)c->Nq * c->nKp * es) + al256((size_t)c->Nk * nw * 8) +
                         al256((size_t)c->Nk * nw * 4) + al256((size_t)c->Nq * nm * 8) + al256((size_t)c->Nq * nm * 4);
    auto per_batch = [&](int64_t nb) {
        return al256((size_t)nb * c->nRge * es) + 2 * al256((size_t)nb * nrow * es) +
               al256((size_t)nb * c->Nq * ncol * es) + al256((size_t)nb * nqblk * per * 8) + al256((size_t)nb * per * 8);
    };
    if (fixed + per_batch(1) > (size_t)PGB_NOALLOC_SCRATCH_BYTES) {
        c->err = "scattering_rates_noalloc: this grid needs " + std::to_string(fixed + per_batch(1)) +
                 " bytes of scratch for one k-point; the fixed scratch holds " +
                 std::to_string((size_t)PGB_NOALLOC_SCRATCH_BYTES);
        return PGB_EINVAL;
    }
    int64_t nbmax = 1;
    while (nbmax < nk && nbmax < 65535 && fixed + per_batch(nbmax + 1) <= (size_t)PGB_NOALLOC_SCRATCH_BYTES) ++nbmax;

    unsigned char *base = nullptr;
    pgb_status st = scratch_address(c, &base);
    if (st != PGB_OK) return st;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += al256(bytes);
        return p;
    };
    int *bad = reinterpret_cast<int *>(take(sizeof(int)));
    float2 *phq = reinterpret_cast<float2 *>(take((size_t)c->Nq * c->nKp * es));
    double *focc = reinterpret_cast<double *>(take((size_t)c->Nk * nw * 8));
    float *eps32 = reinterpret_cast<float *>(take((size_t)c->Nk * nw * 4));
    double *nbe = reinterpret_cast<double *>(take((size_t)c->Nq * nm * 8));
    float *hw32 = reinterpret_cast<float *>(take((size_t)c->Nq * nm * 4));
    char *phk = reinterpret_cast<char *>(take((size_t)nbmax * c->nRge * es));
    char *S1 = reinterpret_cast<char *>(take((size_t)nbmax * nrow * es));
    char *G = reinterpret_cast<char *>(take((size_t)nbmax * nrow * es));
    char *Cb = reinterpret_cast<char *>(take((size_t)nbmax * c->Nq * ncol * es));
    double *partial = reinterpret_cast<double *>(take((size_t)nbmax * nqblk * per * 8));
    double *gmode = reinterpret_cast<double *>(take((size_t)nbmax * per * 8));

    // k indices must lie on the grid (the flag word is the only region cleared)
    {
        int hbad = 0;
        if (cudaMemsetAsync(bad, 0, sizeof(int), c->stream) != cudaSuccess) return PGB_ECUDA;
        k_check_kidx<<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>(k_idx, nk, c->Nk, bad);
        c->launches++;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            c->err = "scattering_rates_noalloc: CUDA error while checking k indices";
            return PGB_ECUDA;
        }
        if (hbad) {
            c->err = "scattering_rates_noalloc: k index out of range";
            return PGB_EINVAL;
        }
    }
    // every other scratch region is fully overwritten before it is read, so
    // nothing else has to be cleared between calls
    if ((st = launch_qtable_grid(c, nullptr, c->Nq, phq, true)) != PGB_OK) return st;
    if ((st = launch_occ_tables(c, T, mu, focc, eps32, nbe, hw32)) != PGB_OK) return st;
    const double scale = kTwoPiOverHbar / ((double)c->Nq * sigma * kSqrtPi);
    for (int64_t b0 = 0; b0 < nk; b0 += nbmax) {
        const int64_t nb = std::min<int64_t>(nbmax, nk - b0);
        const int32_t *kb = k_idx + b0;
        if ((st = launch_phase_grid(c, c->kg, kb, nb, c->d_Rge, c->nRge, phk, true)) != PGB_OK) return st;
        if ((st = launch_cgemm(c, true, 1, nb, nrowS, c->nRge, phk, c->nRge, 0, c->d_g32, nrowS, 0, S1, nrowS, 0)) !=
            PGB_OK)
            return st;
        if ((st = launch_fold_u(c, true, nb, kb, c->nRgp, nm, nw, S1, c->d_U32, G)) != PGB_OK) return st;
        if ((st = launch_cgemm(c, true, nb, c->Nq, ncol, c->nKp, phq, c->nKp, 0, G, ncol, nrow, Cb, ncol,
                               c->Nq * ncol)) != PGB_OK)
            return st;
        RatesArgs ra;
        ra.nb = nb;
        ra.kidx = kb;
        ra.Nq = c->Nq;
        for (int d = 0; d < 3; ++d) {
            ra.kg[d] = c->kg[d];
            ra.qg[d] = c->qg[d];
        }
        ra.nw = nw;
        ra.nm = nm;
        ra.C = Cb;
        ra.U = c->d_U32;
        ra.coef = c->d_coef32;
        ra.eps = c->d_eps;
        ra.hw = c->d_hw;
        ra.T = T;
        ra.mu = mu;
        ra.sigma = sigma;
        ra.eps32 = eps32;
        ra.focc = focc;
        ra.nbe = nbe;
        ra.hw32 = hw32;
        ra.partial = partial;
        ra.nqblk = nqblk;
        ra.qpb = qpb;
        ra.qiters = qiters;
        if ((st = launch_rates_epilogue(c, true, ra)) != PGB_OK) return st;
        if ((st = launch_rates_reduce(c, nb, nqblk, nm, nw, scale, partial, gamma_out + b0 * nw, gmode)) != PGB_OK)
            return st;
    }
    return PGB_OK;
}
