// Helpers shared by the Schur-complement ALC kernels (the FP32-bulk form in
// alc_bulk32.cu, the FP64 Schur form in alc_schur64.cu).
#pragma once
#include <cuda_runtime.h>

#include "device_util.cuh"

namespace alc {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// CPT consecutive values of a candidate-indexed row (vector loads/stores)
template <int CPT, typename T>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[CPT]) {
    if constexpr (sizeof(T) == 4 && CPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 4) {
            float4 t = *reinterpret_cast<const float4 *>(p + r);
            v[r] = t.x;
            v[r + 1] = t.y;
            v[r + 2] = t.z;
            v[r + 3] = t.w;
        }
    } else if constexpr (CPT % 2 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 2) {
            typename Vec2<T>::type t = *reinterpret_cast<const typename Vec2<T>::type *>(p + r);
            v[r] = t.x;
            v[r + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < CPT; r++) v[r] = p[r];
    }
}

template <int CPT, typename T>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[CPT]) {
    if constexpr (sizeof(T) == 4 && CPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 4)
            *reinterpret_cast<float4 *>(p + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
    } else if constexpr (CPT % 2 == 0) {
#pragma unroll
        for (int r = 0; r < CPT; r += 2) {
            typename Vec2<T>::type t;
            t.x = v[r];
            t.y = v[r + 1];
            *reinterpret_cast<typename Vec2<T>::type *>(p + r) = t;
        }
    } else {
#pragma unroll
        for (int r = 0; r < CPT; r++) p[r] = v[r];
    }
}

// Integer key with the order of the doubles (for comparisons off the FP64 pipe)
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// (score, row, slot) argmax across a warp: larger score, ties to the lower row
__device__ __forceinline__ void warp_best3(float &s, int &row, int &slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float os = __shfl_xor_sync(LAGP_FULL_MASK, s, o);
        int orow = __shfl_xor_sync(LAGP_FULL_MASK, row, o);
        int oslot = __shfl_xor_sync(LAGP_FULL_MASK, slot, o);
        if (os > s || (os == s && orow < row)) {
            s = os;
            row = orow;
            slot = oslot;
        }
    }
}

}  // namespace alc
