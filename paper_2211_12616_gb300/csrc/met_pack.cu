// Met snapshot repacking (read_met + "update device", arxiv 2211.12616
// Sections 3.1 and 4.1): variables given as separate [level][lat][lon] float32
// arrays become one record per grid point, [lat][lon][level] x (u, v, omega, T),
// so that the two levels of a cell column are adjacent in memory.
//
// 16-bit storage first reduces each (variable, level) plane to its largest
// magnitude maxabs = m 2^E (m in [0.5, 1)) and stores the power-of-two scale
// 2^(E-15); codes are round-to-nearest-even of x * 2^(15-E), an exact scaling.
//
// The transpose goes through shared memory in tiles of 32 longitudes x 32
// levels: reads are 128-byte rows of one level, writes are runs of 32
// consecutive records.  The same values go to this slot's lane of the
// interleaved pair records that the particle kernels read (two slots per grid
// point), in both pair buffers the slot belongs to; for bf16 the pair records
// hold the stored values with their level scale applied.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace mptrac {
namespace {

constexpr int kTile = 32;

// One block per (variable, level): largest |x| over the lat-lon plane, then
// the power-of-two scale of that plane.
__global__ void k_plane_scale(const float* __restrict__ f0, const float* __restrict__ f1,
                              const float* __restrict__ f2, const float* __restrict__ f3,
                              int64_t plane, int nz, float* scales) {
    const int k = blockIdx.x, var = blockIdx.y;
    const float* f = var == 0 ? f0 : var == 1 ? f1 : var == 2 ? f2 : f3;
    float m = 0.f;
    if (f) {
        const float* row = f + (int64_t)k * plane;
        for (int64_t q = threadIdx.x; q < plane; q += blockDim.x) m = fmaxf(m, fabsf(row[q]));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) {
            float s = 1.f;
            if (m > 0.f) {
                int e;
                frexpf(m, &e);
                s = ldexpf(1.f, e - 15);
            }
            scales[var * nz + k] = s;
        }
    }
}

__device__ __forceinline__ uint32_t code16(float x, int storage) {
    if (storage == MPTRAC_BF16) return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
    return (uint32_t)__half_as_ushort(__float2half_rn(x));
}

// grid (ceil(nx/32), ny, ceil(nz/32)), block (32, 8)
template <int ST>
__global__ void __launch_bounds__(256) k_pack(const float* __restrict__ u, const float* __restrict__ v,
                                              const float* __restrict__ w, const float* __restrict__ T,
                                              int nx, int ny, int nz, void* recv,
                                              const float* __restrict__ scales, void* pairs0, int lane0,
                                              void* pairs1, int lane1) {
    __shared__ float tile[4][kTile][kTile + 1];   // [var][level][lon]
    const int i0 = blockIdx.x * kTile, j = blockIdx.y, k0 = blockIdx.z * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t plane = (int64_t)nx * ny;
    const float* src[4] = {u, v, w, T};
#pragma unroll
    for (int var = 0; var < 4; ++var) {
        for (int kk = ty; kk < kTile; kk += 8) {
            const int k = k0 + kk, i = i0 + tx;
            float x = 0.f;
            if (src[var] && k < nz && i < nx) {
                x = src[var][(int64_t)k * plane + (int64_t)j * nx + i];
                if (ST != MPTRAC_FP32) x *= 1.0f / scales[var * nz + k];
            }
            tile[var][kk][tx] = x;
        }
    }
    __syncthreads();
    const int t = ty * kTile + tx;
#pragma unroll
    for (int rep = 0; rep < (kTile * kTile) / 256; ++rep) {
        const int e = rep * 256 + t;
        const int il = e / kTile, kl = e % kTile;
        const int i = i0 + il, k = k0 + kl;
        if (i >= nx || k >= nz) continue;
        const int64_t r = ((int64_t)j * nx + i) * nz + k;
        // each pair record is rewritten whole (read, replace this slot's lane,
        // write): full-sector accesses instead of four scattered partial ones
        if (ST == MPTRAC_FP32) {
            static_cast<float4*>(recv)[r] =
                make_float4(tile[0][kl][il], tile[1][kl][il], tile[2][kl][il], tile[3][kl][il]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float4* pr = static_cast<float4*>(q ? pairs1 : pairs0) + 2 * r;
                const int lane = q ? lane1 : lane0;
                float4 lo = pr[0], hi = pr[1];   // (u0, u1, v0, v1), (w0, w1, T0, T1)
                if (lane == 0) {
                    lo.x = tile[0][kl][il]; lo.z = tile[1][kl][il]; hi.x = tile[2][kl][il]; hi.z = tile[3][kl][il];
                } else {
                    lo.y = tile[0][kl][il]; lo.w = tile[1][kl][il]; hi.y = tile[2][kl][il]; hi.w = tile[3][kl][il];
                }
                pr[0] = lo;
                pr[1] = hi;
            }
        } else {
            uint32_t c[4];
#pragma unroll
            for (int var = 0; var < 4; ++var) c[var] = code16(tile[var][kl][il], ST);
            static_cast<uint2*>(recv)[r] = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
            if (ST == MPTRAC_BF16) {
                // the pair records hold the stored value itself (code times its power-of-two
                // level scale): bf16 has float32's exponent range, so the product is again a
                // bf16 number (for |value| >= 2^-126) and the step kernel needs no scale
#pragma unroll
                for (int var = 0; var < 4; ++var)
                    c[var] = code16(__uint_as_float(c[var] << 16) * scales[var * nz + k], ST);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint4* pr = static_cast<uint4*>(q ? pairs1 : pairs0) + r;   // words (u, v, omega, T), lane 0 low
                const int lane = q ? lane1 : lane0;
                uint4 w4 = *pr;
                const uint32_t keep = lane == 0 ? 0xFFFF0000u : 0x0000FFFFu;
                const int sh = lane == 0 ? 0 : 16;
                w4.x = (w4.x & keep) | (c[0] << sh);
                w4.y = (w4.y & keep) | (c[1] << sh);
                w4.z = (w4.z & keep) | (c[2] << sh);
                w4.w = (w4.w & keep) | (c[3] << sh);
                *pr = w4;
            }
        }
    }
}

__global__ void k_fill(float* p, int n, float v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

cudaError_t launch_pack(int storage, int nvars, const float* u, const float* v, const float* w,
                        const float* T, int nx, int ny, int nz, void* rec, float* scales, void* pairs0,
                        int lane0, void* pairs1, int lane1, cudaStream_t s) {
    if (nvars < 4) T = nullptr;
    const int64_t plane = (int64_t)nx * ny;
    note_launches(2);
    if (storage == MPTRAC_FP32) {
        k_fill<<<(4 * nz + 255) / 256, 256, 0, s>>>(scales, 4 * nz, 1.f);
    } else {
        k_plane_scale<<<dim3(nz, 4), 512, 0, s>>>(u, v, w, T, plane, nz, scales);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((nx + kTile - 1) / kTile, ny, (nz + kTile - 1) / kTile), block(kTile, 8);
    switch (storage) {
        case MPTRAC_FP32: k_pack<MPTRAC_FP32><<<grid, block, 0, s>>>(u, v, w, T, nx, ny, nz, rec, scales, pairs0, lane0, pairs1, lane1); break;
        case MPTRAC_BF16: k_pack<MPTRAC_BF16><<<grid, block, 0, s>>>(u, v, w, T, nx, ny, nz, rec, scales, pairs0, lane0, pairs1, lane1); break;
        default: k_pack<MPTRAC_FP16><<<grid, block, 0, s>>>(u, v, w, T, nx, ny, nz, rec, scales, pairs0, lane0, pairs1, lane1); break;
    }
    return cudaGetLastError();
}

namespace {
// Copy of n 16-byte elements, `reps` times, loads and stores cached in L2 only.
// Each repetition shifts the block-to-element mapping by one block, and every
// thread keeps four loads in flight before its stores.
__global__ void __launch_bounds__(512) k_copy_probe(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                    int64_t n, int reps) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        const int64_t b = (blockIdx.x + (unsigned)r) % gridDim.x;
        int64_t i = b * blockDim.x + threadIdx.x;
        for (; i + 3 * T < n; i += 4 * T) {
            const uint4 a0 = __ldcg(src + i), a1 = __ldcg(src + i + T);
            const uint4 a2 = __ldcg(src + i + 2 * T), a3 = __ldcg(src + i + 3 * T);
            __stcg(dst + i, a0);
            __stcg(dst + i + T, a1);
            __stcg(dst + i + 2 * T, a2);
            __stcg(dst + i + 3 * T, a3);
        }
        for (; i < n; i += T) __stcg(dst + i, __ldcg(src + i));
    }
}
}  // namespace

cudaError_t launch_copy_probe(const void* src, void* dst, size_t bytes, int reps, int num_sms, cudaStream_t s) {
    note_launches(1);
    k_copy_probe<<<4 * num_sms, 512, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst),
                                             (int64_t)(bytes / 16), reps);
    return cudaGetLastError();
}

}  // namespace mptrac
