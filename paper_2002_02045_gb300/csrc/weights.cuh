// Energy mismatch and Gaussian weight of one scattering term in the fused
// tensor-core epilogue (Sec. 2.1.2, Eqs. scatter_rate and BTE_W), shared with
// the diagnostic entry that checks them against FP64.
//
// Band energies are shifted by a reference e_ref (so every shifted energy is at
// least 1 eV) and, like hbar*omega, held as a (hi, lo) pair of floats whose sum
// carries ~48 significant bits.  For a term that can pass the 7 sigma screen the
// two hi parts are within a factor of two, so their difference is exact; the
// mismatch x = e_n(k) - e_m(k+q) + s hbar*omega (s = -1 emission, +1 absorption)
// then carries only the last two FP32 roundings (|dx| <= 7.5e-9 eV for
// |x| <= 0.1 eV), and the weight exp(-(x/sigma)^2) is taken in FP32.
#pragma once
#include <cuda_runtime.h>

namespace pgb {

// (hi, lo) float pair of a double: hi = fl32(v), lo = fl32(v - hi).
__host__ __device__ __forceinline__ float2 split_hl(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// x from the pair differences dh = e_n,hi - e_m,hi and dl = e_n,lo - e_m,lo.
__device__ __forceinline__ float mismatch32(float dh, float dl, float2 w, float s) {
    return (dh + s * w.x) + (dl + s * w.y);
}

// exp(-(x/sigma)^2), FP32.
__device__ __forceinline__ float gauss32(float x, float inv_sigma) {
    const float y = x * inv_sigma;
    return expf(-y * y);
}

}  // namespace pgb
