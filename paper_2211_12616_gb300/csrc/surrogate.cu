// Learned displacement surrogate: stencil features, BF16 tensor-core MLP
// (forward, backward, Adam) and inference with an envelope test.  The paper
// has no learned component; this is the project's addition on top of the
// advection module (arxiv 2211.12616, Section 3.2).
//
// Network (per sample): x_hat = (x - mu_x)/sd_x (176 = 168 features + 8 zero
// pad), z1 = x_hat W1 + b1, h1 = gelu(z1), z2 = h1 W2 + b2, h2 = gelu(z2),
// y_hat = h2 W3 + b3 (3 outputs, padded to 8 columns), y = y_hat sd_y + mu_y.
// GEMM operands are bfloat16 with float32 accumulation on the 5th-generation
// tensor cores (tcgen05.mma, operands in shared memory, accumulators in tensor
// memory), both in training and in the fused inference; kernels on the
// warp-level mma.sync m16n8k16 stay selectable for comparison.  Biases, GELU,
// the loss and Adam run in float32 on float32 master weights.
#include <cmath>
#include <cstring>

#include "internal.h"
#include "met_record.cuh"

namespace mptrac {
namespace {

constexpr int NF = MPTRAC_SURR_NFEAT, KP = MPTRAC_SURR_KPAD, HID = MPTRAC_SURR_HIDDEN,
              NO = MPTRAC_SURR_NOUT, NOP = 8;
// offsets of the flat parameter vector
constexpr int OW1 = 0, OB1 = OW1 + KP * HID, OW2 = OB1 + HID, OB2 = OW2 + HID * HID,
              OW3 = OB2 + HID, OB3 = OW3 + HID * NO, NPAR = OB3 + NO;
static_assert(NPAR == MPTRAC_SURR_NPARAM, "parameter count");

constexpr double kR = 6371000.0;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// features and targets
// ---------------------------------------------------------------------------
struct FeatArgs {
    Geo g;
    MetView m0, m1;
    int64_t n;
    const double *lon, *lat, *p;
    float w;
    float* X;            // [n][KP]
};

template <int ST>
__global__ void __launch_bounds__(128) k_features(const FeatArgs a) {
    const Geo& g = a.g;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    using R = typename RecT<ST>::T;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const double lon = a.lon[q], lat = a.lat[q], p = a.p[q];
        // nearest node, float64 like the definition
        double r = fmod(lon - g.lon0_d, 360.0);
        if (r < 0.0) r += 360.0;
        const double x = r / g.dlon_d;
        const double xr = floor(x + 0.5);
        long long i0 = (long long)xr % g.nx;
        if (i0 < 0) i0 += g.nx;
        const double y = (lat - g.lat0_d) / g.dlat_d;
        long long j0 = (long long)floor(y + 0.5);
        j0 = j0 < 1 ? 1 : (j0 > g.ny - 2 ? g.ny - 2 : j0);
        const double pc = fmin(fmax(p, g.pmin_d), g.pmax_d);
        int lo = 0, hi = g.nz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (g.plev_d[mid] >= pc) lo = mid + 1; else hi = mid;
        }
        int k = lo - 1;
        k = k < 0 ? 0 : (k > g.nz - 2 ? g.nz - 2 : k);
        double fz = (g.plev_d[k] - pc) / (g.plev_d[k] - g.plev_d[k + 1]);
        fz = fmin(fmax(fz, 0.0), 1.0);
        const double z = k + fz;
        long long k0 = (long long)floor(z + 0.5);
        k0 = k0 < 1 ? 1 : (k0 > g.nz - 2 ? g.nz - 2 : k0);
        float* X = a.X + q * KP;
        const R* rec[2] = {static_cast<const R*>(a.m0.rec), static_cast<const R*>(a.m1.rec)};
        const float* sc[2] = {a.m0.scales, a.m1.scales};
        for (int s = 0; s < 2; ++s) {
            int col = 0;
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = (int)k0 + dk;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int jj = (int)j0 + dj;
                    for (int di = -1; di <= 1; ++di) {
                        int ii = (int)i0 + di;
                        ii = ii < 0 ? ii + g.nx : (ii >= g.nx ? ii - g.nx : ii);
                        float4 v = decode<ST>(__ldg(rec[s] + ((int64_t)jj * g.nx + ii) * g.nz + kk));
                        if (ST != MPTRAC_FP32) {
                            v.x *= sc[s][kk];
                            v.y *= sc[s][g.nz + kk];
                            v.z *= sc[s][2 * g.nz + kk];
                        }
                        X[s * 81 + col] = v.x;
                        X[s * 81 + 27 + col] = v.y;
                        X[s * 81 + 54 + col] = v.z;
                        ++col;
                    }
                }
            }
        }
        // columns: [snapshot][variable][dk][dj][di] (2 x 3 x 27), then the extras
        X[162] = (float)(x - xr);
        X[163] = (float)(y - (double)j0);
        X[164] = (float)(z - (double)k0);
        X[165] = a.w;
        double sn, cs;
        sincos(lat * (kPi / 180.0), &sn, &cs);
        X[166] = (float)sn;
        X[167] = (float)cs;
#pragma unroll
        for (int c = NF; c < KP; ++c) X[c] = 0.f;
    }
}

__global__ void k_targets(int64_t n, const double* lon0, const double* lat0, const double* p0,
                          const double* lon1, const double* lat1, const double* p1, float* Y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        double dl = fmod(lon1[q] - lon0[q] + 180.0, 360.0);
        if (dl < 0.0) dl += 360.0;
        dl -= 180.0;
        const double c = cos(lat0[q] * (kPi / 180.0));
        Y[3 * q + 0] = (float)(kR * c * dl * (kPi / 180.0));
        Y[3 * q + 1] = (float)(kR * (lat1[q] - lat0[q]) * (kPi / 180.0));
        Y[3 * q + 2] = (float)log(p1[q] / p0[q]);
    }
}

// column sums and sums of squares (float partials per block, float64 totals)
__global__ void k_colstats(const float* __restrict__ D, int64_t n, int ncol, int rows_per_block,
                           double* sum, double* sumsq) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        float s = 0.f, s2 = 0.f, comp = 0.f, comp2 = 0.f;
        for (int64_t r = r0; r < r1; ++r) {
            const float v = D[r * ncol + c];
            // compensated summation keeps the float partials accurate
            float yv = v - comp, t = s + yv;
            comp = (t - s) - yv;
            s = t;
            float y2 = v * v - comp2, t2 = s2 + y2;
            comp2 = (t2 - s2) - y2;
            s2 = t2;
        }
        atomicAdd(&sum[c], (double)s);
        atomicAdd(&sumsq[c], (double)s2);
    }
}

// the sums (in mean, sd) -> mean and standard deviation; sd <= sd_min -> 1
__global__ void k_colstats_final(int64_t n, int ncol, double sd_min, double* mean, double* sd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const double m = mean[c] / (double)n;
    const double v = fmax(sd[c] / (double)n - m * m, 0.0);
    const double sdev = sqrt(v);
    mean[c] = m;
    sd[c] = sdev > sd_min ? sdev : 1.0;
}

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM (mma.sync m16n8k16, f32 accumulate) with epilogues
// C[M x N] = A[M x K] * B[K x N]; element (m, k) of A at A[m*sam + k*sak],
// element (k, n) of B at B[k*sbk + n*sbn]; optional split over K.
// ---------------------------------------------------------------------------
enum Epi { EPI_ATOMIC_F32 = 0, EPI_BIAS_GELU = 1, EPI_BIAS_F32 = 2, EPI_GELU_BWD = 3 };

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int64_t M, N, K;
    int64_t sam, sak, sbk, sbn;
    int64_t kchunk;         // K range per blockIdx.z
    // epilogue
    float* Cf;              // f32 output (atomic accumulate / pre-activation / y_hat)
    __nv_bfloat16* Cb;      // bf16 output (activation / gradient)
    const float* bias;
    const float* Zin;       // pre-activation for the GELU derivative
    int64_t ldc;
    int64_t n_valid;        // columns >= n_valid are not written
    int* status;            // tcgen05 kernel: set to 1 when a bounded wait gives up
    long long wait_cycles;  // tcgen05 kernel: limit of each wait (SM clock cycles)
};

// GELU(x) = x Phi(x), Phi the standard normal distribution function, without
// the special-function unit.  For |x| <= 4.5, Phi(x) = 1/2 + x P(z) with
// z = x^2 / 10.125 - 1 in [-1, 1] and P of degree 12; x is clamped to
// [-4.5, 4.5] (beyond, Phi is within 3.4e-6 of 0 or 1).  The coefficients were
// fitted here: least squares on [0, 4.5], reweighted toward equal ripple; the
// error of Phi is below 4.2e-8 with the coefficients rounded to float32 and
// below 1.1e-7 evaluated in float32, the accuracy of 0.5 (1 + erff(x / sqrt 2)).
// Every operation is
// explicitly rounded, so that the scalar form and the packed form (two values
// per instruction, lanes rounding like the scalar instructions) agree bit for bit.
constexpr float kPhiT = 4.5f, kPhiS = 2.0f / (4.5f * 4.5f);

// P(z) by Horner's rule, highest coefficient first (the coefficients of z^12 .. z^0)
__device__ __forceinline__ float phi_poly(float x) {
    const float xc = fminf(fmaxf(x, -kPhiT), kPhiT);
    const float z = __fmaf_rn(xc, __fmul_rn(xc, kPhiS), -1.f);
    float q = 1.186082663e-04f;
    q = __fmaf_rn(q, z, -3.718789958e-04f);
    q = __fmaf_rn(q, z, 6.197711336e-04f);
    q = __fmaf_rn(q, z, -1.314797322e-03f);
    q = __fmaf_rn(q, z, 3.128047800e-03f);
    q = __fmaf_rn(q, z, -6.279318128e-03f);
    q = __fmaf_rn(q, z, 1.122274343e-02f);
    q = __fmaf_rn(q, z, -1.857017539e-02f);
    q = __fmaf_rn(q, z, 2.833536640e-02f);
    q = __fmaf_rn(q, z, -4.018990323e-02f);
    q = __fmaf_rn(q, z, 5.469672382e-02f);
    q = __fmaf_rn(q, z, -7.718981802e-02f);
    q = __fmaf_rn(q, z, 1.569049954e-01f);
    return __fmaf_rn(xc, q, 0.5f);
}
__device__ __forceinline__ float gelu(float x) { return __fmul_rn(x, phi_poly(x)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return phi_poly(x) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Pairs of float32 values in one 64-bit register for Blackwell's packed
// float32x2 instructions (each lane rounds exactly like the scalar instruction).
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(f2_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_dup(float a) { return f2_pack(a, a); }

// gelu of both lanes of x: the same operations as gelu(), two values per instruction
__device__ __forceinline__ f2_t gelu2(f2_t x) {
    float a, b;
    f2_split(x, a, b);
    const f2_t xc = f2_pack(fminf(fmaxf(a, -kPhiT), kPhiT), fminf(fmaxf(b, -kPhiT), kPhiT));
    const f2_t z = f2_fma(xc, f2_mul(xc, f2_dup(kPhiS)), f2_dup(-1.f));
    f2_t q = f2_dup(1.186082663e-04f);
    q = f2_fma(q, z, f2_dup(-3.718789958e-04f));
    q = f2_fma(q, z, f2_dup(6.197711336e-04f));
    q = f2_fma(q, z, f2_dup(-1.314797322e-03f));
    q = f2_fma(q, z, f2_dup(3.128047800e-03f));
    q = f2_fma(q, z, f2_dup(-6.279318128e-03f));
    q = f2_fma(q, z, f2_dup(1.122274343e-02f));
    q = f2_fma(q, z, f2_dup(-1.857017539e-02f));
    q = f2_fma(q, z, f2_dup(2.833536640e-02f));
    q = f2_fma(q, z, f2_dup(-4.018990323e-02f));
    q = f2_fma(q, z, f2_dup(5.469672382e-02f));
    q = f2_fma(q, z, f2_dup(-7.718981802e-02f));
    q = f2_fma(q, z, f2_dup(1.569049954e-01f));
    return f2_mul(x, f2_fma(xc, q, f2_dup(0.5f)));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs& g, int64_t m, int64_t n, float v) {
    if (m >= g.M || n >= g.N || n >= g.n_valid) return;
    const int64_t o = m * g.ldc + n;
    if (EPI == EPI_ATOMIC_F32) {
        atomicAdd(&g.Cf[o], v);
    } else if (EPI == EPI_BIAS_GELU) {
        const float z = v + g.bias[n];
        g.Cf[o] = z;
        g.Cb[o] = __float2bfloat16_rn(gelu(z));
    } else if (EPI == EPI_BIAS_F32) {
        g.Cf[o] = v + g.bias[n];
    } else {
        g.Cb[o] = __float2bfloat16_rn(v * gelu_grad(g.Zin[o]));
    }
}

// The 16 consecutive columns [n, n + 16) of row m (one tensor-memory load of
// the tcgen05 GEMM) through the epilogue: 16-byte loads, stores and atomics
// where the row segment is whole and aligned, else element by element.  The
// arithmetic is that of gemm_epilogue, element for element.
template <int EPI>
__device__ __forceinline__ void gemm_epilogue16(const GemmArgs& g, int64_t m, int64_t n, const float (&v)[16]) {
    if (m >= g.M) return;
    const int64_t o = m * g.ldc + n;
    bool vec = n + 16 <= g.N && n + 16 <= g.n_valid && (g.ldc & 7) == 0 && (n & 7) == 0;
    if (EPI != EPI_GELU_BWD) vec = vec && (reinterpret_cast<uintptr_t>(g.Cf + o) & 15) == 0;
    if (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD) vec = vec && (reinterpret_cast<uintptr_t>(g.Cb + o) & 15) == 0;
    if (EPI == EPI_GELU_BWD) vec = vec && (reinterpret_cast<uintptr_t>(g.Zin + o) & 15) == 0;
    if (!vec) {
#pragma unroll
        for (int j = 0; j < 16; ++j) gemm_epilogue<EPI>(g, m, n + j, v[j]);
        return;
    }
    if (EPI == EPI_ATOMIC_F32) {
        float4* dst = reinterpret_cast<float4*>(g.Cf + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        return;
    }
    float r[16];   // f32 result (BIAS_*) or pre-activation (GELU_BWD)
    if (EPI == EPI_GELU_BWD) {
        const float4* zin = reinterpret_cast<const float4*>(g.Zin + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 z = zin[q];
            r[4 * q] = z.x;
            r[4 * q + 1] = z.y;
            r[4 * q + 2] = z.z;
            r[4 * q + 3] = z.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = v[j] + g.bias[n + j];
        float4* dst = reinterpret_cast<float4*>(g.Cf + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
    if (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD) {
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float a = EPI == EPI_BIAS_GELU ? gelu(r[2 * j]) : v[2 * j] * gelu_grad(r[2 * j]);
            const float b = EPI == EPI_BIAS_GELU ? gelu(r[2 * j + 1]) : v[2 * j + 1] * gelu_grad(r[2 * j + 1]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            w[j] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* dst = reinterpret_cast<uint4*>(g.Cb + o);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

constexpr int TM = 64, TN = 64, TK = 32, TKP = TK + 8;

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
    __shared__ __nv_bfloat16 As[TM][TKP];   // [m][k]
    __shared__ __nv_bfloat16 Bs[TN][TKP];   // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;          // 2 x 2 warps, 32 x 32 each
    const int gq = lane >> 2, tq = lane & 3;
    const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;
    const int64_t kb0 = (int64_t)blockIdx.z * g.kchunk;
    const int64_t kend = min(g.K, kb0 + g.kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    const bool a_mfast = g.sam == 1, b_nfast = g.sbn == 1;
    for (int64_t kb = kb0; kb < kend; kb += TK) {
        for (int e = tid; e < TM * TK; e += 128) {
            const int r = a_mfast ? (e % TM) : (e / TK), c = a_mfast ? (e / TM) : (e % TK);
            const int64_t m = m0 + r, k = kb + c;
            As[r][c] = (m < g.M && k < kend) ? g.A[m * g.sam + k * g.sak] : zero;
        }
        for (int e = tid; e < TN * TK; e += 128) {
            const int r = b_nfast ? (e % TN) : (e / TK), c = b_nfast ? (e / TN) : (e % TK);
            const int64_t n = n0 + r, k = kb + c;
            Bs[r][c] = (n < g.N && k < kend) ? g.B[k * g.sbk + n * g.sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + gq;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int nn = wn * 32 + j * 8 + gq;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[nn][kk + 2 * tq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[nn][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    // epilogue: c0,c1 -> (row gq, cols 2tq, 2tq+1); c2,c3 -> (row gq+8, same cols)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t m = m0 + wm * 32 + i * 16 + gq + (c >> 1) * 8;
                const int64_t n = n0 + wn * 32 + j * 8 + 2 * tq + (c & 1);
                gemm_epilogue<EPI>(g, m, n, acc[i][j][c]);
            }
}

// x_hat = bf16((x - mu)/sd), zero pad; one warp per row; env[row] = max |x_hat| <= 4
__global__ void k_normalise(const float* __restrict__ X, int64_t n, const float* mu, const float* isd,
                            __nv_bfloat16* Xh, uint8_t* env) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float mx = 0.f;
    for (int c = lane; c < KP; c += 32) {
        float v = 0.f;
        if (c < NF) {
            v = (X[row * KP + c] - mu[c]) * isd[c];
            mx = fmaxf(mx, fabsf(v));
        }
        Xh[row * KP + c] = __float2bfloat16_rn(v);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (env && lane == 0) env[row] = (mx <= 4.f) ? 1 : 0;
}

// loss = mean (y_hat - t_hat)^2 over the 3 outputs; dY = 2 (y_hat - t_hat)/(3B) (bf16, 8 columns);
// db3 += column sums of the bf16 dY (the operand the W3 gradient uses), summed in float32
__global__ void k_loss(const float* __restrict__ Yh, const float* __restrict__ Yt, int64_t B,
                       const float* mu_y, const float* isd_y, __nv_bfloat16* dY, float* loss, float* db3) {
    __shared__ float red[4][32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float l = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    const float scale = 2.f / (3.f * (float)B);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < B; q += stride) {
        float dd[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const float r = Yh[q * NOP + j] - (Yt[q * NO + j] - mu_y[j]) * isd_y[j];
            l += r * r;
            const __nv_bfloat16 g = __float2bfloat16_rn(scale * r);
            dd[j] = __bfloat162float(g);
            dY[q * NOP + j] = g;
        }
#pragma unroll
        for (int j = NO; j < NOP; ++j) dY[q * NOP + j] = __float2bfloat16(0.f);
        d0 += dd[0];
        d1 += dd[1];
        d2 += dd[2];
    }
    float v[4] = {l, d0, d1, d2};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float x = v[c];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) red[c][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float x = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x += red[threadIdx.x][i];
        if (threadIdx.x == 0) atomicAdd(loss, x / (3.f * (float)B));
        else atomicAdd(&db3[threadIdx.x - 1], x);
    }
}

// out[c] += sum over rows of D[row][c] (bf16 input), c < 128
__global__ void k_colsum_bf16(const __nv_bfloat16* __restrict__ D, int64_t n, int rows_per_block, float* out) {
    const int c = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
    float s = 0.f;
    for (int64_t r = r0; r < r1; ++r) s += __bfloat162float(D[r * HID + c]);
    atomicAdd(&out[c], s);
}

// Adam (Kingma & Ba) on the float32 master parameters, then the bf16 weight copies
__global__ void k_adam(float* theta, const float* grad, float* m, float* v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_cast_weights(const float* theta, __nv_bfloat16* W1b, __nv_bfloat16* W2b,
                               __nv_bfloat16* W3b, float* b3p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < KP * HID) W1b[i] = __float2bfloat16_rn(theta[OW1 + i]);
    if (i < HID * HID) W2b[i] = __float2bfloat16_rn(theta[OW2 + i]);
    if (i < HID * NOP) {
        const int r = i / NOP, c = i % NOP;
        W3b[i] = __float2bfloat16_rn(c < NO ? theta[OW3 + r * NO + c] : 0.f);
    }
    if (i < NOP) b3p[i] = i < NO ? theta[OB3 + i] : 0.f;
}

// ---------------------------------------------------------------------------
// Fused inference: stencil gather -> standardise (shared memory, bf16) ->
// three tensor-core layers -> displacement, for tiles of 128 particles.
// 256 threads: in the gather each (particle, snapshot) pair has one thread;
// in the MLP each warp owns 16 rows of the tile through all three layers, so
// the layers need no block-wide barrier; the weights stay in shared memory
// for the whole (persistent) launch.
// ---------------------------------------------------------------------------
constexpr int FT = 128;                 // particles per tile
constexpr int XS = KP + 8, HS = HID + 8;  // padded row strides (bf16 elements): conflict-free fragments

struct FusedArgs {
    Geo g;
    MetView m0, m1;
    int64_t n;
    double *lon, *lat, *p;
    uint8_t* fallback;
    float w;
    int window_ok;
    const __nv_bfloat16 *W1b, *W2b, *W3b;
    const float *b1, *b2, *b3p, *mu_x, *isd_x, *mu_y, *sd_y;
    double lon0, pmin, pmax;
    int* status;            // set to 1 when a bounded wait of the tcgen05 kernel gives up
    long long wait_cycles;  // limit of each wait for the tensor cores (SM clock cycles)
    int withhold_mma;       // test hook: issue no MMA (nothing completes, the wait runs out)
    unsigned long long* fb_count;   // if not null: the number of fallback particles is added here
};

constexpr size_t kFusedSmem = (size_t)HID * XS * 2 + (size_t)HID * HS * 2 + (size_t)NOP * HS * 2 +
                              (size_t)(2 * HID + NOP) * 4 + (size_t)2 * KP * 4 + (size_t)FT * XS * 2 +
                              (size_t)FT * HS * 2 + (size_t)FT * NOP * 4 + FT * 4 + (size_t)kMaxNZ * 4;

// Nearest node in float32 (latitude in float-float): used by the fused
// inference, where a different choice within ~1e-6 cells of a half-cell
// boundary only swaps one valid stencil for its neighbour.  Level search from
// the float level table.
__device__ __forceinline__ void nearest_node_f32(const Geo& g, const float* plev, double lon, double lat,
                                                 double p, int& i0, int& j0, int& k0, float& ox, float& oy,
                                                 float& oz) {
    float lf = (float)(lon - (double)g.lon0);
    if (lf < 0.f) lf += 360.f;
    if (lf >= 360.f) lf -= 360.f;
    const float x = lf * g.inv_dlon;
    const float xr = floorf(x + 0.5f);
    int ii = (int)xr;
    if (ii >= g.nx) ii -= g.nx;
    ii = min(max(ii, 0), g.nx - 1);
    const float lat_hi = (float)lat, lat_lo = (float)(lat - (double)lat_hi);
    const float y = ((lat_hi - g.lat0) + lat_lo) * g.inv_dlat;
    int jj = (int)floorf(y + 0.5f);
    jj = min(max(jj, 1), g.ny - 2);
    const float pc = fminf(fmaxf((float)p, g.pmin), g.pmax);
    int lo = 0, hi = g.nz;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (plev[mid] >= pc) lo = mid + 1; else hi = mid;
    }
    int k = min(max(lo - 1, 0), g.nz - 2);
    const float fz = fminf(fmaxf((plev[k] - pc) / (plev[k] - plev[k + 1]), 0.f), 1.f);
    const float z = (float)k + fz;
    int kk = (int)floorf(z + 0.5f);
    kk = min(max(kk, 1), g.nz - 2);
    i0 = ii;
    j0 = jj;
    k0 = kk;
    ox = x - xr;
    oy = y - (float)jj;
    oz = z - (float)kk;
}

struct Pos {
    double lon, lat, p;
};

// Position of particle q (zeros past n).
__device__ __forceinline__ Pos pos_of(const FusedArgs& a, int64_t q) {
    if (q >= a.n) return Pos{0.0, 0.0, 0.0};
    return Pos{a.lon[q], a.lat[q], a.p[q]};
}

// Position of the particle of (particle, snapshot) item `tid` of tile `tile`.
__device__ __forceinline__ Pos load_pos(const FusedArgs& a, int64_t tile, int tid) {
    return pos_of(a, tile * FT + (tid >> 1));
}

// The predicted displacement of particle q at position `pos` (normalised
// outputs y0..y2) followed by the position rules, or the fallback flag outside
// the envelope.
__device__ __forceinline__ void apply_displacement(const FusedArgs& a, int64_t q, const Pos& pos, int env_ok,
                                                   float y0, float y1, float y2) {
    const double la = pos.lat;
    const bool ok = a.window_ok && env_ok && fabs(la) <= 80.0;
    a.fallback[q] = ok ? 0 : 1;
    if (a.fb_count) {   // the lanes of the warp that flag a fallback, counted with one atomic
        const unsigned act = __activemask();
        const unsigned fb = __ballot_sync(act, !ok);
        if (fb && (int)(threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(a.fb_count, (unsigned long long)__popc(fb));
    }
    if (!ok) return;
    const float dx = y0 * a.sd_y[0] + a.mu_y[0];
    const float dy = y1 * a.sd_y[1] + a.mu_y[1];
    const float dz = y2 * a.sd_y[2] + a.mu_y[2];
    const float cl = cospif((float)la * (1.0f / 180.0f));
    double lo = pos.lon + (double)(dx / ((float)kR * cl) * (float)(180.0 / kPi));
    double lt = la + (double)(dy * (float)(180.0 / (kPi * kR)));
    const double pp = pos.p * (double)expf(dz);
    if (lt > 90.0) { lt = 180.0 - lt; lo += 180.0; }
    else if (lt < -90.0) { lt = -180.0 - lt; lo += 180.0; }
    if (lo >= a.lon0 + 360.0) lo -= 360.0;
    if (lo < a.lon0) lo += 360.0;
    a.lon[q] = lo;
    a.lat[q] = lt;
    a.p[q] = fmin(fmax(pp, a.pmin), a.pmax);
}

// Gather and standardisation of one tile: thread = (particle pl, snapshot sn)
// at position `pos` reads the 27 stencil records of its snapshot and stores the
// standardised bf16 features through xs(row, column, value); env[row] = every
// standardised feature within +-4 (rows past n: zero features, env 0).
template <int ST, class XStore>
__device__ __forceinline__ void gather_standardise(const FusedArgs& a, const float* plevs, const float* mu,
                                                   const float* isd, int64_t tile, int tid, Pos pos, XStore xs,
                                                   int* env) {
    const Geo& g = a.g;
    using R = typename RecT<ST>::T;
    const int pl = tid >> 1, sn = tid & 1;
    const int64_t q = tile * FT + pl;
    float mx = 0.f;
    if (q < a.n) {
        int i0, j0, k0;
        float ox, oy, oz;
        const double lat = pos.lat;
        nearest_node_f32(g, plevs, pos.lon, lat, pos.p, i0, j0, k0, ox, oy, oz);
        const R* rec = static_cast<const R*>(sn ? a.m1.rec : a.m0.rec);
        const float* sc = sn ? a.m1.scales : a.m0.scales;
        int im = i0 - 1, ip = i0 + 1;
        if (im < 0) im += g.nx;
        if (ip >= g.nx) ip -= g.nx;
        const int icol[3] = {im, i0, ip};
        R r[27];
#pragma unroll
        for (int c = 0; c < 27; ++c) {
            const int dk = c / 9 - 1, dj = (c / 3) % 3 - 1, di = c % 3;
            r[c] = __ldg(rec + ((int64_t)(j0 + dj) * g.nx + icol[di]) * g.nz + (k0 + dk));
        }
#pragma unroll
        for (int c = 0; c < 27; ++c) {
            float4 v = decode<ST>(r[c]);
            if (ST != MPTRAC_FP32) {
                const int kk = k0 + c / 9 - 1;
                v.x *= sc[kk];
                v.y *= sc[g.nz + kk];
                v.z *= sc[2 * g.nz + kk];
            }
            const int c0 = sn * 81 + c;
            const float xu = (v.x - mu[c0]) * isd[c0];
            const float xv = (v.y - mu[c0 + 27]) * isd[c0 + 27];
            const float xw = (v.z - mu[c0 + 54]) * isd[c0 + 54];
            mx = fmaxf(mx, fmaxf(fabsf(xu), fmaxf(fabsf(xv), fabsf(xw))));
            xs(pl, c0, __float2bfloat16_rn(xu));
            xs(pl, c0 + 27, __float2bfloat16_rn(xv));
            xs(pl, c0 + 54, __float2bfloat16_rn(xw));
        }
        if (sn == 0) {
            float snl, csl;
            sincospif((float)lat * (1.0f / 180.0f), &snl, &csl);
            const float ex[6] = {ox, oy, oz, a.w, snl, csl};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float xe = (ex[c] - mu[162 + c]) * isd[162 + c];
                mx = fmaxf(mx, fabsf(xe));
                xs(pl, 162 + c, __float2bfloat16_rn(xe));
            }
#pragma unroll
            for (int c = NF; c < KP; ++c) xs(pl, c, __float2bfloat16(0.f));
        }
    } else {
        for (int c = sn; c < KP; c += 2) xs(pl, c, __float2bfloat16(0.f));
        mx = 1e30f;
    }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    if (sn == 0) env[pl] = (mx <= 4.f) ? 1 : 0;
}

template <int ST>
__global__ void __launch_bounds__(256, 1) k_surr_fused(const FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W1T = reinterpret_cast<__nv_bfloat16*>(smem);            // [HID][XS]
    __nv_bfloat16* W2T = W1T + HID * XS;                                      // [HID][HS]
    __nv_bfloat16* W3T = W2T + HID * HS;                                      // [NOP][HS]
    float* bias = reinterpret_cast<float*>(W3T + NOP * HS);                   // b1 | b2 | b3
    float* mu = bias + 2 * HID + NOP;                                         // [KP]
    float* isd = mu + KP;                                                     // [KP]
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(isd + KP);          // [FT][XS]
    __nv_bfloat16* Hs = Xs + FT * XS;                                         // [FT][HS]
    float* Ys = reinterpret_cast<float*>(Hs + FT * HS);                       // [FT][NOP]
    int* env = reinterpret_cast<int*>(Ys + FT * NOP);                         // [FT]
    float* plevs = reinterpret_cast<float*>(env + FT);                        // [nz]
    const int tid = threadIdx.x;
    for (int e = tid; e < a.g.nz; e += blockDim.x) plevs[e] = a.g.plev[e];
    for (int e = tid; e < KP * HID; e += blockDim.x) {
        const int k = e / HID, nn = e % HID;
        W1T[nn * XS + k] = a.W1b[e];
    }
    for (int e = tid; e < HID * HID; e += blockDim.x) {
        const int k = e / HID, nn = e % HID;
        W2T[nn * HS + k] = a.W2b[e];
    }
    for (int e = tid; e < HID * NOP; e += blockDim.x) {
        const int k = e / NOP, nn = e % NOP;
        W3T[nn * HS + k] = a.W3b[e];
    }
    for (int e = tid; e < HID; e += blockDim.x) {
        bias[e] = a.b1[e];
        bias[HID + e] = a.b2[e];
    }
    if (tid < NOP) bias[2 * HID + tid] = a.b3p[tid];
    for (int e = tid; e < KP; e += blockDim.x) {
        mu[e] = a.mu_x[e];
        isd[e] = a.isd_x[e];
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, gq = lane >> 2, tq = lane & 3;
    const int64_t ntiles = (a.n + FT - 1) / FT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        gather_standardise<ST>(a, plevs, mu, isd, tile, tid, load_pos(a, tile, tid),
                               [&](int r, int c, __nv_bfloat16 v) { Xs[r * XS + c] = v; }, env);
        __syncthreads();
        // ---- MLP: warp owns rows r0 .. r0+15 ----
        const int r0 = warp * 16;
        {
            float acc[16][4];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < KP; kk += 16) {
                uint32_t af[4];
                af[0] = *reinterpret_cast<const uint32_t*>(&Xs[(r0 + gq) * XS + kk + 2 * tq]);
                af[1] = *reinterpret_cast<const uint32_t*>(&Xs[(r0 + gq + 8) * XS + kk + 2 * tq]);
                af[2] = *reinterpret_cast<const uint32_t*>(&Xs[(r0 + gq) * XS + kk + 2 * tq + 8]);
                af[3] = *reinterpret_cast<const uint32_t*>(&Xs[(r0 + gq + 8) * XS + kk + 2 * tq + 8]);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    uint32_t bf[2];
                    bf[0] = *reinterpret_cast<const uint32_t*>(&W1T[(8 * j + gq) * XS + kk + 2 * tq]);
                    bf[1] = *reinterpret_cast<const uint32_t*>(&W1T[(8 * j + gq) * XS + kk + 2 * tq + 8]);
                    mma_bf16(acc[j], af, bf);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = r0 + gq + (c >> 1) * 8, col = 8 * j + 2 * tq + (c & 1);
                    Hs[row * HS + col] = __float2bfloat16_rn(gelu(acc[j][c] + bias[col]));
                }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < HID; kk += 16) {
                uint32_t af[4];
                af[0] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq) * HS + kk + 2 * tq]);
                af[1] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq + 8) * HS + kk + 2 * tq]);
                af[2] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq) * HS + kk + 2 * tq + 8]);
                af[3] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq + 8) * HS + kk + 2 * tq + 8]);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    uint32_t bf[2];
                    bf[0] = *reinterpret_cast<const uint32_t*>(&W2T[(8 * j + gq) * HS + kk + 2 * tq]);
                    bf[1] = *reinterpret_cast<const uint32_t*>(&W2T[(8 * j + gq) * HS + kk + 2 * tq + 8]);
                    mma_bf16(acc[j], af, bf);
                }
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = r0 + gq + (c >> 1) * 8, col = 8 * j + 2 * tq + (c & 1);
                    Hs[row * HS + col] = __float2bfloat16_rn(gelu(acc[j][c] + bias[HID + col]));
                }
            __syncwarp();
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < HID; kk += 16) {
                uint32_t af[4], bf[2];
                af[0] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq) * HS + kk + 2 * tq]);
                af[1] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq + 8) * HS + kk + 2 * tq]);
                af[2] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq) * HS + kk + 2 * tq + 8]);
                af[3] = *reinterpret_cast<const uint32_t*>(&Hs[(r0 + gq + 8) * HS + kk + 2 * tq + 8]);
                bf[0] = *reinterpret_cast<const uint32_t*>(&W3T[gq * HS + kk + 2 * tq]);
                bf[1] = *reinterpret_cast<const uint32_t*>(&W3T[gq * HS + kk + 2 * tq + 8]);
                mma_bf16(o, af, bf);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int row = r0 + gq + (c >> 1) * 8, col = 2 * tq + (c & 1);
                Ys[row * NOP + col] = o[c] + bias[2 * HID + col];
            }
        }
        __syncthreads();
        // ---- apply the displacement (or flag the particle for the fallback) ----
        if (tid < FT) {
            const int64_t q = tile * FT + tid;
            if (q < a.n)
                apply_displacement(a, q, pos_of(a, q), env[tid], Ys[tid * NOP + 0], Ys[tid * NOP + 1],
                                   Ys[tid * NOP + 2]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Fused inference on the 5th-generation tensor cores.  Same gather and
// standardisation; then each layer of the 128-particle tile is one chain of
// tcgen05.mma (M = 128 particles; N = 128, 128, 16; K = 176, 128, 128 in steps
// of 16) issued by one thread, with both operands in shared memory in the
// K-major core-matrix layout without swizzle and the accumulator in tensor
// memory.  The block is split by role: warps 0-3 (consumers) run the layers --
// the MMA chains, and the epilogues that read the accumulators with tcgen05.ld
// (warp w reads the 32 lanes 32 w + 0..31, every column), add the bias, apply
// GELU and write the next layer's operand in place of the tile's input, which
// the first layer has consumed -- while warps 4-11 (producers) gather and
// standardise the next tile into the other of two input buffers.  Full/empty
// mbarriers hand the buffers over, so the stencil gather of one tile overlaps
// the layers of the one before.  Every wait (for
// a buffer or for the MMA completion) is bounded in time; when one gives up
// the kernel raises an abort flag that every other wait also watches, sets
// *status, stops, frees its tensor memory and returns.
// ---------------------------------------------------------------------------
constexpr int KG1 = KP / 8, KG2 = HID / 8;   // core-matrix columns of the K = 176 and K = 128 operands
constexpr int NW3 = 16;                      // layer 3: the 3 outputs padded to N = 16
constexpr uint32_t kTmemCols = 256;          // layer 1 in columns 0..127, layer 2 in 128..255, layer 3 in 0..15
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at the SM clock
constexpr long long kTestWaitCycles = 20000000LL;  // ~10 ms: the wait test hook
constexpr int kTcConsumers = 128, kTcProducers = 256, kTcThreads = kTcConsumers + kTcProducers;
constexpr int kConsumerBar = 1;              // named barrier of the consumer warps (0 is __syncthreads)

constexpr size_t kTcW1 = (size_t)HID * KP * 2, kTcW2 = (size_t)HID * HID * 2, kTcW3 = (size_t)NW3 * HID * 2,
                 kTcX = (size_t)FT * KP * 2, kTcH = (size_t)FT * HID * 2;
constexpr size_t kTcSmem = kTcW1 + kTcW2 + kTcW3 + 2 * kTcX + (size_t)(2 * HID + NOP) * 4 +
                           (size_t)2 * KP * 4 + (size_t)2 * FT * 4 + (size_t)kMaxNZ * 4 + 64;
static_assert(kTcW1 % 128 == 0 && kTcW2 % 128 == 0 && kTcW3 % 128 == 0 && kTcX % 128 == 0 && kTcH % 128 == 0,
              "operand blocks keep 128-byte alignment");
static_assert(kTcSmem <= 227 * 1024, "shared memory of the tcgen05 inference kernel");
static_assert(kTcH <= kTcX, "the hidden activations fit in place of the tile's input");

// Byte offset of element (row r, column k) of a bf16 operand stored as 8 x 8
// core matrices of 128 contiguous bytes (8 rows of 16 bytes), core matrix
// (r / 8, k / 8) at ((r / 8) kg + k / 8) 128: the K-direction core matrices of
// a row group are adjacent (128 bytes apart), row groups kg * 128 bytes apart.
__device__ __forceinline__ uint32_t cm_off(int r, int k, int kg) {
    return (uint32_t)(((((r >> 3) * kg) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between the core matrices adjacent in K), stride-dimension byte
// offset (between adjacent 8-row groups), all in 16-byte units; descriptor
// version 1; no swizzle, base offset 0.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: float32 accumulator, bf16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// One layer: D (tensor memory) = A (M x K) * B^T (B stored N x K), K in steps
// of 16 = two core matrices along K (128 bytes apart; row groups kg * 128).
__device__ __forceinline__ void umma_layer(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, int ksteps, int kg,
                                           uint32_t idesc) {
    const uint32_t lbo = 128u, sbo = (uint32_t)kg * 128u;
    for (int ks = 0; ks < ksteps; ++ks)
        umma_f16(d_tmem, umma_desc(a_addr + 256u * ks, lbo, sbo), umma_desc(b_addr + 256u * ks, lbo, sbo), idesc,
                 ks > 0 ? 1u : 0u);
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for phase `phase` of the mbarrier, for at most `limit` SM cycles; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// mbar_wait that also gives up as soon as another thread of the block has raised *abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t phase, long long limit,
                                                   const volatile int* abort) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if (*abort || clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Named barrier over `n` threads that also ORs a predicate over them: every
// participant gets the same answer, so a decision to stop stays uniform.
__device__ __forceinline__ bool bar_red_or(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// 16 consecutive float32 accumulator columns of this thread's lane.  The wait
// names the registers, so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without its wait, and the wait that names the 16 registers it
// fills (so that no use is scheduled before it): a load can run while the
// previous chunk is computed.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])::"memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 accumulator values of columns [c, c + 16) + bias, GELU, bf16, into the next
// layer's A operand at row `row`.
__device__ __forceinline__ void gelu_chunk(const uint32_t* v, int row, int c, const float* bias, unsigned char* Hs) {
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const f2_t bb = *reinterpret_cast<const f2_t*>(bias + c + 2 * i);
        float lo, hi;
        f2_split(gelu2(f2_add(f2_pack(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1])), bb)), lo, hi);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
        pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    *reinterpret_cast<uint4*>(Hs + cm_off(row, c, KG2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(Hs + cm_off(row, c + 8, KG2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Epilogue of layers 1 and 2 for a whole row: the 128 accumulator columns of
// this thread's lane, in chunks of 16; the load of each chunk runs while the
// one before is computed (two register buffers, a loop of two chunks).
__device__ __forceinline__ void tc_epilogue_gelu_row(uint32_t taddr, int row, const float* bias, unsigned char* Hs) {
    uint32_t r0[16], r1[16];
    tmem_ld16_issue(taddr, r0);
    tmem_ld_wait(r0);
#pragma unroll 1
    for (int k = 0; k < HID / 32; ++k) {
        const int c = 32 * k;
        tmem_ld16_issue(taddr + (uint32_t)(c + 16), r1);
        gelu_chunk(r0, row, c, bias, Hs);
        tmem_ld_wait(r1);
        if (k + 1 < HID / 32) tmem_ld16_issue(taddr + (uint32_t)(c + 32), r0);
        gelu_chunk(r1, row, c + 16, bias, Hs);
        if (k + 1 < HID / 32) tmem_ld_wait(r0);
    }
}

template <int ST>
__global__ void __launch_bounds__(kTcThreads, 1) k_surr_fused_tc(const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* W1s = tc_smem;                    // B of layer 1: [HID][KP] core matrices
    unsigned char* W2s = W1s + kTcW1;                // B of layer 2: [HID][HID]
    unsigned char* W3s = W2s + kTcW2;                // B of layer 3: [16][HID] (rows 3..15 zero)
    unsigned char* Xs0 = W3s + kTcW3;                // A of layer 1 ([FT][KP]), then of layers 2 and 3
                                                     // ([FT][HID]): two buffers
    float* bias = reinterpret_cast<float*>(Xs0 + 2 * kTcX);     // b1 | b2 | b3
    float* mu = bias + 2 * HID + NOP;                            // [KP]
    float* isd = mu + KP;                                        // [KP]
    int* env = reinterpret_cast<int*>(isd + KP);                 // [2][FT]
    float* plevs = reinterpret_cast<float*>(env + 2 * FT);       // [kMaxNZ]
    uint64_t* bars = reinterpret_cast<uint64_t*>(plevs + kMaxNZ);   // full[2], empty[2], mma
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    const volatile int* vabort = abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t full_b[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
    const uint32_t empty_b[2] = {smem_u32(&bars[2]), smem_u32(&bars[3])};
    const uint32_t mma_b = smem_u32(&bars[4]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full_b[b]), "r"(kTcProducers) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty_b[b]), "r"(kTcConsumers) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mma_b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    for (int e = tid; e < a.g.nz; e += blockDim.x) plevs[e] = a.g.plev[e];
    // weights as B operands (N x K, K-major): W1 [k][n] -> (n, k)
    for (int e = tid; e < KP * HID; e += blockDim.x) {
        const int k = e / HID, nn = e % HID;
        *reinterpret_cast<__nv_bfloat16*>(W1s + cm_off(nn, k, KG1)) = a.W1b[e];
    }
    for (int e = tid; e < HID * HID; e += blockDim.x) {
        const int k = e / HID, nn = e % HID;
        *reinterpret_cast<__nv_bfloat16*>(W2s + cm_off(nn, k, KG2)) = a.W2b[e];
    }
    for (int e = tid; e < NW3 * HID; e += blockDim.x) {
        const int nn = e / HID, k = e % HID;
        *reinterpret_cast<__nv_bfloat16*>(W3s + cm_off(nn, k, KG2)) =
            nn < NOP ? a.W3b[k * NOP + nn] : __float2bfloat16(0.f);
    }
    for (int e = tid; e < HID; e += blockDim.x) {
        bias[e] = a.b1[e];
        bias[HID + e] = a.b2[e];
    }
    if (tid < NOP) bias[2 * HID + tid] = a.b3p[tid];
    for (int e = tid; e < KP; e += blockDim.x) {
        mu[e] = a.mu_x[e];
        isd[e] = a.isd_x[e];
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const int64_t ntiles = (a.n + FT - 1) / FT;

    if (warp >= kTcConsumers / 32) {
        // ---- producers: gather and standardise tile i into buffer i mod 2 ----
        const int pt = tid - kTcConsumers;   // (particle, snapshot) item pt of the tile
        int i = 0;
        // the positions of the next tile are loaded while this one is gathered (the consumers
        // write positions only of tiles the producers are done with)
        Pos next = blockIdx.x < ntiles ? load_pos(a, blockIdx.x, pt) : Pos{0.0, 0.0, 0.0};
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            const Pos pos = next;
            if (tile + gridDim.x < ntiles) next = load_pos(a, tile + gridDim.x, pt);
            if (i >= 2) {   // the consumers are done with tile i - 2 in this buffer
                const bool ok = mbar_wait_or_abort(empty_b[b], (uint32_t)(((i >> 1) - 1) & 1), a.wait_cycles, vabort);
                if (__any_sync(0xffffffffu, !ok)) {
                    *abort_flag = 1;
                    break;
                }
            }
            unsigned char* X = Xs0 + b * kTcX;
            auto xs = [&](int r, int c, __nv_bfloat16 v) { *reinterpret_cast<__nv_bfloat16*>(X + cm_off(r, c, KG1)) = v; };
            gather_standardise<ST>(a, plevs, mu, isd, tile, pt, pos, xs, env + b * FT);
            fence_async_smem();   // the tensor cores read what the generic stores wrote
            mbar_arrive(full_b[b]);
        }
    } else {
        // ---- consumers: the three layers of tile i and the displacement ----
        const int row = tid;
        const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
        const uint32_t w1_a = smem_u32(W1s), w2_a = smem_u32(W2s), w3_a = smem_u32(W3s);
        uint32_t phase = 0;
        bool failed = false;
        int i = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ok_in = mbar_wait_or_abort(full_b[b], (uint32_t)((i >> 1) & 1), a.wait_cycles, vabort);
            if (bar_red_or(kConsumerBar, kTcConsumers, !ok_in)) {
                failed = true;
                break;
            }
            unsigned char* Xb = Xs0 + b * kTcX;
            const uint32_t xs_a = smem_u32(Xb);   // the input, then (after layer 1) the hidden activations
            const Pos mine = pos_of(a, tile * FT + row);   // read now, used after the third layer
#pragma unroll 1
            for (int layer = 0; layer < 3; ++layer) {
                if (layer > 0) {   // this layer's operand, written by every consumer, reaches the tensor cores
                    fence_async_smem();
                    tc_fence_before();
                    bar_sync_n(kConsumerBar, kTcConsumers);
                }
                if (tid == 0 && !a.withhold_mma) {
                    tc_fence_after();
                    if (layer == 0)
                        umma_layer(tbase, xs_a, w1_a, KP / 16, KG1, umma_idesc(FT, HID));
                    else if (layer == 1)
                        umma_layer(tbase + 128u, xs_a, w2_a, HID / 16, KG2, umma_idesc(FT, HID));
                    else
                        umma_layer(tbase, xs_a, w3_a, HID / 16, KG2, umma_idesc(FT, NW3));
                    umma_commit(mma_b);
                }
                const bool ok = mbar_wait_or_abort(mma_b, phase, a.wait_cycles, vabort);
                phase ^= 1u;
                if (bar_red_or(kConsumerBar, kTcConsumers, !ok)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                if (layer == 0) {
                    tc_epilogue_gelu_row(tlane, row, bias, Xb);
                } else if (layer == 1) {
                    tc_epilogue_gelu_row(tlane + 128u, row, bias + HID, Xb);
                } else {
                    float y[4];
                    tmem_ld4(tlane, y);
                    const int64_t q = tile * FT + row;
                    if (q < a.n)
                        apply_displacement(a, q, mine, env[b * FT + row], y[0] + bias[2 * HID],
                                           y[1] + bias[2 * HID + 1], y[2] + bias[2 * HID + 2]);
                }
            }
            if (failed) break;
            // every accumulator read of this tile is done before the next tile's MMAs overwrite
            // them; the input buffer and its envelope flags go back to the producers
            tc_fence_before();
            bar_sync_n(kConsumerBar, kTcConsumers);
            mbar_arrive(empty_b[b]);
        }
        if (failed) *abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *vabort) atomicExch(a.status, 1);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Training GEMM on tcgen05: CTA tile 128 x 128 (M x N), K in chunks of 64 held
// in two shared-memory stages (A and B of a chunk in the K-major core-matrix
// layout, written by all threads from any strides), four MMAs of K = 16 per
// chunk issued by one thread and committed to the stage's mbarrier, so that the
// loads of chunk i + 1 overlap the MMAs of chunk i.  The accumulator (128
// lanes x 128 columns of tensor memory) goes through the same epilogues as
// k_gemm.  Waits are bounded as in k_surr_fused_tc.
// ---------------------------------------------------------------------------
constexpr int GT_M = 128, GT_K = 64;   // the tile's N (BN) is 128, or 64 where M alone gives few tiles
template <int BN>
__host__ __device__ constexpr size_t gemm_stage_bytes() { return (size_t)(GT_M + BN) * GT_K * 2; }   // 32 KB (BN 128), 24 KB (64)
template <int BN>
__host__ __device__ constexpr size_t gemm_tc_smem() { return 2 * gemm_stage_bytes<BN>() + 32; }

// Rows [r0, r0 + ROWS) x columns [kb, kb + GT_K) of an operand whose element
// (row, k) is P[row * s_row + k * s_k], into the core-matrix layout at dst;
// rows >= nrows and k >= kend are zero.  16-byte loads along k when k is
// contiguous, along the rows when the rows are, else element by element.
template <int ROWS>
__device__ __forceinline__ void load_operand(unsigned char* dst, const __nv_bfloat16* P, int64_t s_row, int64_t s_k,
                                             int64_t r0, int64_t nrows, int64_t kb, int64_t kend, int tid) {
    const bool aligned = (reinterpret_cast<uintptr_t>(P) & 15) == 0;
    if (aligned && s_k == 1 && (s_row & 7) == 0 && (kend & 7) == 0) {
        for (int e = tid; e < ROWS * (GT_K / 8); e += 256) {
            const int r = e / (GT_K / 8), c = 8 * (e % (GT_K / 8));
            const int64_t row = r0 + r, k = kb + c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < nrows && k < kend) v = *reinterpret_cast<const uint4*>(P + row * s_row + k);
            *reinterpret_cast<uint4*>(dst + cm_off(r, c, GT_K / 8)) = v;
        }
    } else if (aligned && s_row == 1 && (s_k & 7) == 0 && (nrows & 7) == 0) {
        for (int e = tid; e < (ROWS / 8) * GT_K; e += 256) {
            const int r = 8 * (e % (ROWS / 8)), c = e / (ROWS / 8);
            const int64_t row = r0 + r, k = kb + c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < nrows && k < kend) v = *reinterpret_cast<const uint4*>(P + row + k * s_k);
            const unsigned short* h = reinterpret_cast<const unsigned short*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<unsigned short*>(dst + cm_off(r + j, c, GT_K / 8)) = h[j];
        }
    } else {
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        for (int e = tid; e < ROWS * GT_K; e += 256) {
            const int r = e / GT_K, c = e % GT_K;
            const int64_t row = r0 + r, k = kb + c;
            *reinterpret_cast<__nv_bfloat16*>(dst + cm_off(r, c, GT_K / 8)) =
                (row < nrows && k < kend) ? P[row * s_row + k * s_k] : zero;
        }
    }
}

template <int EPI, int BN>
__global__ void __launch_bounds__(256, 1) k_gemm_tc(const GemmArgs g) {
    static_assert(BN == 64 || BN == 128, "tile N of 64 or 128");
    constexpr size_t kGStage = gemm_stage_bytes<BN>();
    constexpr uint32_t kGemmTmemCols = BN;   // a power of two >= 32
    extern __shared__ __align__(128) unsigned char g_smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(g_smem + 2 * kGStage);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t m0 = (int64_t)blockIdx.x * GT_M, n0 = (int64_t)blockIdx.y * BN;
    const int64_t kb0 = (int64_t)blockIdx.z * g.kchunk;
    const int64_t kend = min(g.K, kb0 + g.kchunk);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kGemmTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const int nchunks = kend > kb0 ? (int)((kend - kb0 + GT_K - 1) / GT_K) : 0;
    uint32_t waits0 = 0u, waits1 = 0u;   // completed waits per stage: the parity of the next
    bool failed = false;
    for (int i = 0; i < nchunks; ++i) {
        const int st = i & 1;
        if (i >= 2) {   // the MMAs of chunk i - 2 have read this stage
            const bool ok = mbar_wait(smem_u32(&mbar[st]), (st ? waits1 : waits0) & 1u, g.wait_cycles);
            if (st) ++waits1; else ++waits0;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        unsigned char* As = g_smem + st * kGStage;
        unsigned char* Bs = As + (size_t)GT_M * GT_K * 2;
        const int64_t kb = kb0 + (int64_t)i * GT_K;
        load_operand<GT_M>(As, g.A, g.sam, g.sak, m0, g.M, kb, kend, tid);
        load_operand<BN>(Bs, g.B, g.sbn, g.sbk, n0, g.N, kb, kend, tid);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a_addr = smem_u32(As), b_addr = smem_u32(Bs);
#pragma unroll
            for (int ks = 0; ks < GT_K / 16; ++ks)
                umma_f16(tbase, umma_desc(a_addr + 256u * ks, 128u, 128u * (GT_K / 8)),
                         umma_desc(b_addr + 256u * ks, 128u, 128u * (GT_K / 8)), umma_idesc(GT_M, BN),
                         (i > 0 || ks > 0) ? 1u : 0u);
            umma_commit(smem_u32(&mbar[st]));
        }
    }
    // drain: every commit of both stages has arrived (the last one covers every MMA)
#pragma unroll
    for (int st = 0; st < 2; ++st) {
        const uint32_t commits = (uint32_t)((nchunks + 1 - st) / 2);
        uint32_t& waits = st ? waits1 : waits0;
        while (!failed && waits < commits) {
            const bool ok = mbar_wait(smem_u32(&mbar[st]), waits & 1u, g.wait_cycles);
            ++waits;
            if (__syncthreads_or(!ok)) failed = true;
        }
    }
    if (!failed && nchunks > 0) {
        tc_fence_after();
        const int row = 32 * (warp & 3) + (tid & 31);
        const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ++ch) {   // warps 0-3: columns [0, BN/2), warps 4-7: the rest
            const int c = (BN / 2) * (warp >> 2) + 16 * ch;
            if (n0 + c >= g.N) break;   // warp-uniform
            float v[16];
            tmem_ld16(tlane + (uint32_t)c, v);
            gemm_epilogue16<EPI>(g, m0 + row, n0 + c, v);
        }
    }
    if (failed && tid == 0) atomicExch(g.status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kGemmTmemCols)
                     : "memory");
    }
}

int grid1(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

template <int EPI, int BN>
cudaError_t gemm_tc_bn(const GemmArgs& a, int gz, cudaStream_t s) {
    dim3 grid((unsigned)((a.M + GT_M - 1) / GT_M), (unsigned)((a.N + BN - 1) / BN), (unsigned)std::max(gz, 1));
    note_launches(1);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_tc_smem<BN>());
    if (e != cudaSuccess) return e;
    k_gemm_tc<EPI, BN><<<grid, 256, gemm_tc_smem<BN>(), s>>>(a);
    return cudaGetLastError();
}

// Tiles of 128 x 128, or 128 x 64 where N is at most 64 or where the 128-wide
// tiles would leave more than half the SMs idle (the forward GEMMs of a batch).
template <int EPI>
cudaError_t gemm_tc(const GemmArgs& g, int splits, int* status, cudaStream_t s) {
    GemmArgs a = g;
    a.status = status;
    a.wait_cycles = kWaitCycles;
    if (splits < 1) splits = 1;
    a.kchunk = ((g.K + splits - 1) / splits + GT_K - 1) / GT_K * GT_K;
    if (a.kchunk <= 0) a.kchunk = GT_K;
    const int gz = (int)((g.K + a.kchunk - 1) / a.kchunk);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = 1;
    }
    const int64_t tiles = ((g.M + GT_M - 1) / GT_M) * ((g.N + 127) / 128) * (int64_t)std::max(gz, 1);
    if (g.N <= 64 || 2 * tiles <= sms) return gemm_tc_bn<EPI, 64>(a, gz, s);
    return gemm_tc_bn<EPI, 128>(a, gz, s);
}

template <int EPI>
cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t s) {
    GemmArgs a = g;
    if (splits < 1) splits = 1;
    a.kchunk = ((g.K + splits - 1) / splits + TK - 1) / TK * TK;
    if (a.kchunk <= 0) a.kchunk = TK;
    const int gz = (int)((g.K + a.kchunk - 1) / a.kchunk);
    dim3 grid((unsigned)((g.M + TM - 1) / TM), (unsigned)((g.N + TN - 1) / TN), (unsigned)std::max(gz, 1));
    note_launches(1);
    k_gemm<EPI><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// model object
// ---------------------------------------------------------------------------
cudaError_t surr_alloc(Surrogate& S, int64_t B) {
    S.max_batch = B;
    void** ptrs[] = {(void**)&S.theta, (void**)&S.grad, (void**)&S.m, (void**)&S.v, (void**)&S.W1b,
                     (void**)&S.W2b, (void**)&S.W3b, (void**)&S.b3p, (void**)&S.mu_x, (void**)&S.isd_x,
                     (void**)&S.mu_y, (void**)&S.isd_y, (void**)&S.sd_y, (void**)&S.Xh, (void**)&S.H1,
                     (void**)&S.H2, (void**)&S.dY, (void**)&S.dZ2, (void**)&S.dZ1, (void**)&S.Z1,
                     (void**)&S.Z2, (void**)&S.Yh, (void**)&S.Xraw, (void**)&S.env, (void**)&S.loss_tmp,
                     (void**)&S.status};
    const size_t sizes[] = {NPAR * 4, NPAR * 4, NPAR * 4, NPAR * 4, KP * HID * 2, HID * HID * 2, HID * NOP * 2,
                            NOP * 4, KP * 4, KP * 4, NOP * 4, NOP * 4, NOP * 4, (size_t)B * KP * 2,
                            (size_t)B * HID * 2, (size_t)B * HID * 2, (size_t)B * NOP * 2,
                            (size_t)B * HID * 2, (size_t)B * HID * 2, (size_t)B * HID * 4,
                            (size_t)B * HID * 4, (size_t)B * NOP * 4, (size_t)B * KP * 4, (size_t)B, 16, 16};
    for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
        cudaError_t e = cudaMalloc(ptrs[i], sizes[i]);
        if (e != cudaSuccess) return e;
        e = cudaMemset(*ptrs[i], 0, sizes[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void surr_free(Surrogate& S) {
    void* ptrs[] = {S.theta, S.grad, S.m, S.v, S.W1b, S.W2b, S.W3b, S.b3p, S.mu_x, S.isd_x, S.mu_y,
                    S.isd_y, S.sd_y, S.Xh, S.H1, S.H2, S.dY, S.dZ2, S.dZ1, S.Z1, S.Z2, S.Yh, S.Xraw,
                    S.env, S.loss_tmp, S.status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

cudaError_t surr_cast(Surrogate& S, cudaStream_t s) {
    note_launches(1);
    k_cast_weights<<<grid1(KP * HID, 256), 256, 0, s>>>(S.theta, S.W1b, S.W2b, S.W3b, S.b3p);
    return cudaGetLastError();
}

// The training GEMMs on the kernel the surrogate selects (tcgen05 unless mma.sync is chosen).
template <int EPI>
cudaError_t run_gemm(const Surrogate& S, const GemmArgs& g, int splits, cudaStream_t s) {
    return S.kernel == MPTRAC_SURR_KERNEL_MMA_SYNC ? gemm<EPI>(g, splits, s) : gemm_tc<EPI>(g, splits, S.status, s);
}

// Forward of B rows of raw features X (device, [B][KP]) into S.Yh (normalised outputs).
cudaError_t surr_forward(Surrogate& S, const float* X, int64_t B, cudaStream_t s) {
    note_launches(1);
    k_normalise<<<grid1(B * 32, 256), 256, 0, s>>>(X, B, S.mu_x, S.isd_x, S.Xh, S.env);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GemmArgs g{};
    g.A = S.Xh; g.B = S.W1b; g.M = B; g.N = HID; g.K = KP;
    g.sam = KP; g.sak = 1; g.sbk = HID; g.sbn = 1;
    g.Cf = S.Z1; g.Cb = S.H1; g.bias = S.theta + OB1; g.ldc = HID; g.n_valid = HID;
    if ((e = run_gemm<EPI_BIAS_GELU>(S, g, 1, s)) != cudaSuccess) return e;
    g.A = S.H1; g.B = S.W2b; g.K = HID; g.sam = HID;
    g.Cf = S.Z2; g.Cb = S.H2; g.bias = S.theta + OB2;
    if ((e = run_gemm<EPI_BIAS_GELU>(S, g, 1, s)) != cudaSuccess) return e;
    g.A = S.H2; g.B = S.W3b; g.N = NOP; g.sbk = NOP;
    g.Cf = S.Yh; g.Cb = nullptr; g.bias = S.b3p; g.ldc = NOP; g.n_valid = NOP;
    return run_gemm<EPI_BIAS_F32>(S, g, 1, s);
}

// Split of K (the batch) of a weight-gradient GEMM [M x N]: about one CTA of
// 128 x 128 per SM, each split at least one 64-wide chunk of K.
int wgrad_splits(int64_t M, int64_t N, int64_t B) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = 1;
    }
    const int64_t tiles = ((M + 127) / 128) * ((N + 127) / 128);
    const int64_t want = std::max<int64_t>(1, (int64_t)sms / tiles);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (B + 63) / 64));
}

// Gradients of the loss for B samples into S.grad (zeroed first); loss added to *loss.
cudaError_t surr_backward(Surrogate& S, const float* Yt, int64_t B, float* loss, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(S.grad, 0, NPAR * 4, s);
    if (e != cudaSuccess) return e;
    note_launches(1);
    k_loss<<<grid1(B, 256), 256, 0, s>>>(S.Yh, Yt, B, S.mu_y, S.isd_y, S.dY, loss, S.grad + OB3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmArgs g{};
    // dW3 = H2^T dY  [HID x NO]
    g.A = S.H2; g.sam = 1; g.sak = HID; g.B = S.dY; g.sbk = NOP; g.sbn = 1;
    g.M = HID; g.N = NOP; g.K = B; g.Cf = S.grad + OW3; g.ldc = NO; g.n_valid = NO;
    if ((e = run_gemm<EPI_ATOMIC_F32>(S, g, wgrad_splits(g.M, g.N, B), s)) != cudaSuccess) return e;
    // dZ2 = (dY W3^T) * gelu'(Z2)
    g = GemmArgs{};
    g.A = S.dY; g.sam = NOP; g.sak = 1; g.B = S.W3b; g.sbk = 1; g.sbn = NOP;
    g.M = B; g.N = HID; g.K = NOP; g.Cb = S.dZ2; g.Zin = S.Z2; g.ldc = HID; g.n_valid = HID;
    if ((e = run_gemm<EPI_GELU_BWD>(S, g, 1, s)) != cudaSuccess) return e;
    // dW2 = H1^T dZ2, db2
    g = GemmArgs{};
    g.A = S.H1; g.sam = 1; g.sak = HID; g.B = S.dZ2; g.sbk = HID; g.sbn = 1;
    g.M = HID; g.N = HID; g.K = B; g.Cf = S.grad + OW2; g.ldc = HID; g.n_valid = HID;
    if ((e = run_gemm<EPI_ATOMIC_F32>(S, g, wgrad_splits(g.M, g.N, B), s)) != cudaSuccess) return e;
    const int rpb = 64;   // 128 blocks for a batch of 8192
    note_launches(1);
    k_colsum_bf16<<<grid1(B, rpb), HID, 0, s>>>(S.dZ2, B, rpb, S.grad + OB2);
    // dZ1 = (dZ2 W2^T) * gelu'(Z1)
    g = GemmArgs{};
    g.A = S.dZ2; g.sam = HID; g.sak = 1; g.B = S.W2b; g.sbk = 1; g.sbn = HID;
    g.M = B; g.N = HID; g.K = HID; g.Cb = S.dZ1; g.Zin = S.Z1; g.ldc = HID; g.n_valid = HID;
    if ((e = run_gemm<EPI_GELU_BWD>(S, g, 1, s)) != cudaSuccess) return e;
    // dW1 = Xh^T dZ1, db1
    g = GemmArgs{};
    g.A = S.Xh; g.sam = 1; g.sak = KP; g.B = S.dZ1; g.sbk = HID; g.sbn = 1;
    g.M = KP; g.N = HID; g.K = B; g.Cf = S.grad + OW1; g.ldc = HID; g.n_valid = HID;
    if ((e = run_gemm<EPI_ATOMIC_F32>(S, g, wgrad_splits(g.M, g.N, B), s)) != cudaSuccess) return e;
    note_launches(1);
    k_colsum_bf16<<<grid1(B, rpb), HID, 0, s>>>(S.dZ1, B, rpb, S.grad + OB1);
    return cudaGetLastError();
}

cudaError_t surr_adam(Surrogate& S, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    note_launches(1);
    k_adam<<<grid1(NPAR, 256), 256, 0, s>>>(S.theta, S.grad, S.m, S.v, NPAR, lr, b1, b2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return surr_cast(S, s);
}

cudaError_t launch_surr_features(int storage, const Geo& g, MetView m0, MetView m1, int64_t n,
                                 const double* lon, const double* lat, const double* p, float w,
                                 float* X, cudaStream_t s) {
    FeatArgs a{g, m0, m1, n, lon, lat, p, w, X};
    note_launches(1);
    const int grid = grid1(n, 128);
    switch (storage) {
        case MPTRAC_FP32: k_features<MPTRAC_FP32><<<grid, 128, 0, s>>>(a); break;
        case MPTRAC_BF16: k_features<MPTRAC_BF16><<<grid, 128, 0, s>>>(a); break;
        default: k_features<MPTRAC_FP16><<<grid, 128, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_surr_targets(int64_t n, const double* lon0, const double* lat0, const double* p0,
                                const double* lon1, const double* lat1, const double* p1, float* Y,
                                cudaStream_t s) {
    note_launches(1);
    k_targets<<<grid1(n, 256), 256, 0, s>>>(n, lon0, lat0, p0, lon1, lat1, p1, Y);
    return cudaGetLastError();
}

cudaError_t launch_colstats(const float* D, int64_t n, int ncol, double* mean, double* sd, double sd_min,
                            cudaStream_t s) {
    const int rpb = 2048;
    cudaError_t e = cudaMemsetAsync(mean, 0, (size_t)ncol * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd, 0, (size_t)ncol * sizeof(double), s);
    if (e != cudaSuccess) return e;
    note_launches(2);
    k_colstats<<<grid1(n, rpb), 256, 0, s>>>(D, n, ncol, rpb, mean, sd);
    k_colstats_final<<<(ncol + 255) / 256, 256, 0, s>>>(n, ncol, sd_min, mean, sd);
    return cudaGetLastError();
}

template <class K>
cudaError_t launch_dyn(K kern, int grid, int threads, size_t smem, const FusedArgs& a, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_surr_fused_st(int kernel, int grid, const FusedArgs& a, cudaStream_t s) {
    if (kernel == MPTRAC_SURR_KERNEL_MMA_SYNC) return launch_dyn(k_surr_fused<ST>, grid, 256, kFusedSmem, a, s);
    FusedArgs t = a;
    t.withhold_mma = kernel == MPTRAC_SURR_KERNEL_WAIT_TEST ? 1 : 0;
    t.wait_cycles = t.withhold_mma ? kTestWaitCycles : kWaitCycles;
    return launch_dyn(k_surr_fused_tc<ST>, grid, kTcThreads, kTcSmem, t, s);
}

cudaError_t launch_surr_fused(int storage, Surrogate& S, const Geo& g, MetView m0, MetView m1, int64_t n,
                              double* lon, double* lat, double* p, float w, int window_ok, uint8_t* fallback,
                              uint64_t* fallback_count, double lon0, cudaStream_t s) {
    FusedArgs a{g, m0, m1, n, lon, lat, p, fallback, w, window_ok, S.W1b, S.W2b, S.W3b,
                S.theta + OB1, S.theta + OB2, S.b3p, S.mu_x, S.isd_x, S.mu_y, S.sd_y,
                lon0, g.pmin_d, g.pmax_d, S.status, kWaitCycles, 0,
                reinterpret_cast<unsigned long long*>(fallback_count)};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (n + FT - 1) / FT;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms));
    note_launches(1);
    switch (storage) {
        case MPTRAC_FP32: return launch_surr_fused_st<MPTRAC_FP32>(S.kernel, grid, a, s);
        case MPTRAC_BF16: return launch_surr_fused_st<MPTRAC_BF16>(S.kernel, grid, a, s);
        default: return launch_surr_fused_st<MPTRAC_FP16>(S.kernel, grid, a, s);
    }
}



}  // namespace mptrac
