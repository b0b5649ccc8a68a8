// Met record types and decoding, shared by the kernels that read met slots.
// A record holds (u, v, omega, T) of one grid point: four float32 values, or
// four 16-bit codes (bfloat16 or float16 bit patterns) to be multiplied by the
// per-(level, variable) scale of the slot.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace mptrac {

template <int ST> struct RecT;
template <> struct RecT<MPTRAC_FP32> { using T = float4; };
template <> struct RecT<MPTRAC_BF16> { using T = uint2; };
template <> struct RecT<MPTRAC_FP16> { using T = uint2; };

template <int ST> __device__ __forceinline__ float4 decode(typename RecT<ST>::T r);
template <> __device__ __forceinline__ float4 decode<MPTRAC_FP32>(float4 r) { return r; }
template <> __device__ __forceinline__ float4 decode<MPTRAC_BF16>(uint2 r) {
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u),
                       __uint_as_float(r.y << 16), __uint_as_float(r.y & 0xFFFF0000u));
}
template <> __device__ __forceinline__ float4 decode<MPTRAC_FP16>(uint2 r) {
    return make_float4(__half2float(__ushort_as_half((unsigned short)(r.x & 0xFFFFu))),
                       __half2float(__ushort_as_half((unsigned short)(r.x >> 16))),
                       __half2float(__ushort_as_half((unsigned short)(r.y & 0xFFFFu))),
                       __half2float(__ushort_as_half((unsigned short)(r.y >> 16))));
}


}  // namespace mptrac
