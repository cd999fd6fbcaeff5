// Complex helpers on CUDA's float2 / double2 (x = real, y = imaginary).
#pragma once
#include <cuda_runtime.h>

namespace pgb {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using V2 = typename Vec2<T>::type;

template <typename T>
__host__ __device__ __forceinline__ V2<T> cmake(T re, T im) {
    V2<T> r;
    r.x = re;
    r.y = im;
    return r;
}
template <typename T2>
__host__ __device__ __forceinline__ T2 cadd(T2 a, T2 b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename T2>
__host__ __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc += a * b
template <typename T2>
__host__ __device__ __forceinline__ void cfma(T2 &acc, T2 a, T2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T2>
__host__ __device__ __forceinline__ void cfma_conj(T2 &acc, T2 a, T2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <typename T2>
__host__ __device__ __forceinline__ T2 cconj(T2 a) {
    a.y = -a.y;
    return a;
}
template <typename T2>
__host__ __device__ __forceinline__ auto cabs2(T2 a) -> decltype(a.x) {
    return a.x * a.x + a.y * a.y;
}

}  // namespace pgb
