// Particle kernels of the transport hot path: 4D interpolation, explicit
// midpoint advection on the sphere, Philox-driven turbulent and mesoscale
// diffusion, release masking and position boundary rules
// (module_timesteps / module_advection / module_diffusion_turb /
//  module_diffusion_meso / module_position of arxiv 2211.12616, Sections 3.2
//  and 4.3; the numerics are the readings stated in include/mptrac.h).
//
// GB300 design:
//  * one thread per particle, grid-stride; the particle's state stays in
//    registers for all steps of a launch (temporal blocking), so the particle
//    stream costs ~60 B per launch, not per step;
//  * positions are float64 in memory but carried as float-float pairs
//    (hi + lo) in registers: GB300's float64 rate is a small fraction of its
//    float32 rate;
//  * the 8 corners x 2 snapshots of a particle's current cell stay in
//    registers (or shared memory) as packed float32x2 pairs and are gathered
//    again only when the particle changes cell -- with one 32-byte load per
//    corner from the interleaved pair records, [lat][lon][level] x (u, v,
//    omega, T) x (slot 0, slot 1), whose registers are already the pairs;
//  * random numbers are generated in registers (counter-based Philox): no
//    random-number arrays are stored or read;
//  * divisions and square roots that only scale increments use the hardware
//    approximations (__fdividef: 2 ulp, sqrt.approx), far inside the
//    tolerance.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "cell_key.cuh"
#include "internal.h"
#include "met_record.cuh"

namespace mptrac {
namespace {

constexpr float kCosFloor = 1.745329243e-05f;   // cos(89.999 deg)
constexpr int kMaxDevices = 64;                  // per-device caches of the launchers

// ---------------------------------------------------------------------------
// float-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2)
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(double d) {
    float h = __double2float_rn(d);
    float l = __double2float_rn(d - (double)h);
    return {h, l};
}
__device__ __forceinline__ double ff_val(ff a) { return (double)a.hi + (double)a.lo; }

// a + b with the rounding error of the hi sum carried into lo (Knuth TwoSum),
// then renormalised.  Explicit _rn intrinsics keep the compiler from fusing.
__device__ __forceinline__ ff ff_add(ff a, float b) {
    float s = __fadd_rn(a.hi, b);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    float lo = __fadd_rn(a.lo, e);
    float hi = __fadd_rn(s, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return {hi, lo};
}

// a + b for an increment b no larger than the value (|b| <= |a.hi|), the
// step's case: the error of the hi sum by Fast2Sum (Dekker), exact under that
// condition, then renormalised.  Where |b| > |a.hi| (a longitude just above
// lon0, a latitude just above the south pole) the error term is off by at most
// half an ulp of b, about 1e-9 degrees on a step's increment.
__device__ __forceinline__ ff ff_add_inc(ff a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a.hi));
    float lo = __fadd_rn(a.lo, e);
    const float hi = __fadd_rn(s, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return {hi, lo};
}
// The same sum left unnormalised (|lo| may reach an ulp of hi): enough for a
// position that only places a wind evaluation (the midpoint), 2 fewer operations.
__device__ __forceinline__ ff ff_add_inc_raw(ff a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a.hi));
    return {s, __fadd_rn(a.lo, e)};
}
__device__ __forceinline__ bool ff_less(ff a, float bh, float bl) {
    return a.hi < bh || (a.hi == bh && a.lo < bl);
}
__device__ __forceinline__ bool ff_greater(ff a, float bh, float bl) {
    return a.hi > bh || (a.hi == bh && a.lo > bl);
}

// sin(x) for |x| <= pi/2 as x q(x^2), q of degree 4 with q(0) = 1, in Horner
// form.  The other four coefficients minimise the largest relative error of
// sin(x)/x on [0, pi/2] (a weighted least-squares fit whose weights grow where
// the error is largest, iterated): 1e-8 with the coefficients rounded to
// float32.  Evaluated in float32 the relative error stays below 1.5e-7, that
// of the Taylor series through x^13 in float32, with two fewer multiply-adds.
__device__ __forceinline__ float sin_poly(float x) {
    const float x2 = x * x;
    float q = 2.605783266e-06f;
    q = fmaf(q, x2, -1.980960369e-04f);
    q = fmaf(q, x2, 8.333066478e-03f);
    q = fmaf(q, x2, -1.666665971e-01f);
    q = fmaf(q, x2, 1.0f);
    return x * q;
}

// |cos(lat)| floored at cos(89.999 deg), for the latitude d + inc with d =
// lat - lat0 (float-float) and a float increment inc.  It is the sine of the
// colatitude, formed from the pole's d so that it keeps its relative
// precision next to the poles (the difference with the pole's hi part is
// exact there).
__device__ __forceinline__ float coslat(ff d, float inc, const Geo& g) {
    float colat = (__fadd_rn(d.hi, inc) >= g.dmid)
                      ? __fsub_rn(__fadd_rn(__fsub_rn(g.dn, d.hi), __fsub_rn(g.dn_lo, d.lo)), inc)
                      : __fadd_rn(__fadd_rn(__fsub_rn(d.hi, g.ds), __fsub_rn(d.lo, g.ds_lo)), inc);
    colat = fminf(fmaxf(colat, -90.f), 90.f);
    const float c = fabsf(sin_poly(colat * 0.017453292519943295f));
    return fmaxf(c, kCosFloor);
}

// Reflection of d = lat - lat0 over a pole with d = P (float-float):
// d' = 2 P - d, longitude + 180.  The hi difference is exact (d.hi lies
// within a factor 2 of 2 P.hi next to the pole), the lo parts are renormalised.
__device__ __forceinline__ void reflect(ff& d, float ph, float pl) {
    const float h = __fsub_rn(2.f * ph, d.hi);
    const float l = __fsub_rn(2.f * pl, d.lo);
    d.hi = __fadd_rn(h, l);
    d.lo = __fsub_rn(l, __fsub_rn(d.hi, h));
}

// module_position on (e = lon - lon0, d = lat - lat0, p): reflect over the
// poles (longitude + 180), wrap e into [0, 360), clamp p to the level range.
// The hi parts decide whether any rule can apply; the exact float-float
// comparisons run only then.
__device__ __forceinline__ void horizontal_rules(ff& e, ff& d, const Geo& g) {
    if (ff_greater(d, g.dn, g.dn_lo)) {
        reflect(d, g.dn, g.dn_lo);
        e = ff_add(e, 180.f);
    } else if (ff_less(d, g.ds, g.ds_lo)) {
        reflect(d, g.ds, g.ds_lo);
        e = ff_add(e, 180.f);
    }
    if (!ff_less(e, 360.f, 0.f) || ff_less(e, 0.f, 0.f)) {
        float turns = floorf(e.hi * (1.0f / 360.0f));
        if (isfinite(turns)) {
            e = ff_add(e, -360.f * turns);
            if (!ff_less(e, 360.f, 0.f)) e = ff_add(e, -360.f);
            if (ff_less(e, 0.f, 0.f)) e = ff_add(e, 360.f);
        }
    }
}

__device__ __forceinline__ void position_rules(ff& e, ff& d, ff& p, const Geo& g) {
    horizontal_rules(e, d, g);
    if (ff_less(p, g.pmin, g.pmin_lo)) { p.hi = g.pmin; p.lo = g.pmin_lo; }
    if (ff_greater(p, g.pmax, g.pmax_lo)) { p.hi = g.pmax; p.lo = g.pmax_lo; }
}

__device__ __forceinline__ void position_bc(ff& e, ff& d, ff& p, const Geo& g) {
    // NaN fails every comparison and also takes the exact path (which leaves it)
    if (!(d.hi < g.dn && d.hi > g.ds && e.hi < 360.f && e.hi > 0.f && p.hi > g.pmin && p.hi < g.pmax))
        position_rules(e, d, p, g);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals
// ---------------------------------------------------------------------------
// 32 x 32 -> 64-bit product as one instruction (both halves of the round's
// multiplications from a single multiply)
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    unsigned long long p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c.x, hi0, lo0);
        mul_wide(0xCD9E8D57u, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Philox4x32-10 of the counter (id, step, stream, release) under the key
// schedule taken from the launch arguments (round r uses ks[2r], ks[2r + 1]),
// entered after round 0.  Round 0 multiplies the id word, which does not change
// with the step, and the stream word, a constant (0 or 1): its state is
// (step ^ ks[0], lo(M1 stream), hi(M0 id) ^ release ^ ks[1], lo(M0 id)), whose
// last two words (r0z, r0w) are formed once per particle.
__device__ __forceinline__ uint4 philox_after_round0(uint32_t step, uint32_t stream, uint32_t r0z, uint32_t r0w,
                                                     const uint32_t* ks) {
    uint4 c = make_uint4(step ^ ks[0], stream ? 0xCD9E8D57u : 0u, r0z, r0w);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c.x, hi0, lo0);
        mul_wide(0xCD9E8D57u, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ ks[2 * r], lo1, hi0 ^ c.w ^ ks[2 * r + 1], lo0);
    }
    return c;
}

// Box-Muller pair from two words, z = -r (cos th, sin th) with r^2 = -2 ln u_a
// and th = 2 pi (u_b - 1/2).  A word's top 23 bits m give the uniform
// (m + 1/2) 2^-23 in (0, 1) as F - (1 - 2^-24), F = 1 + m 2^-23 the float with
// exponent 0 and mantissa m; the difference (2m + 1) 2^-24 has at most 24
// significant bits, so it is exact, and so is t = 1 - u_a.  r^2 comes from the hardware
// log2 where u_a >= 1 - 2^-6 does not hold (relative error ~1e-7 there) and
// from the series 2 (t + t^2/2 + t^3/3 + t^4/4) of -2 ln(1 - t) below that
// (truncation < t^5/5 relative, < 2e-8); the factor 2 sits in the
// coefficients, which doubles every rounded step exactly.  The angle is one
// multiply-add on F_b, 2 pi F_b - 2 pi (3/2 - 2^-24), in (-pi, pi) where the
// hardware sine/cosine have absolute error < 4e-7; its own rounding adds
// < 1e-6.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float Fa = __uint_as_float(0x3F800000u | (a >> 9));
    const float Fb = __uint_as_float(0x3F800000u | (b >> 9));
    const float ua = __fsub_rn(Fa, 0.999999940395355224609375f);
    const float t = __fsub_rn(1.0f, ua);
    float r2;
    if (t < 0.015625f)
        r2 = t * fmaf(t, fmaf(t, fmaf(t, 0.5f, 0.66666666666666667f), 1.0f), 2.0f);
    else
        r2 = __log2f(ua) * -1.3862943611198906f;
    const float r = r2 * rsqrtf(r2);
    const float th = fmaf(6.2831853071795865f, Fb, -9.424777586262351f);
    float sn, cs;
    __sincosf(th, &sn, &cs);
    z0 = -r * cs;
    z1 = -r * sn;
}

// ---------------------------------------------------------------------------
// Met record access
// ---------------------------------------------------------------------------

// Shared-memory tables of one block.  NSC = kMaxNZ holds the scales of
// 16-bit storage; float32 storage needs none (NSC = 1, unused).
template <int NSC>
struct SmemT {
    float plev[kMaxNZ];
    float4 lv[kMaxNZ];     // level k: (plev[k], plev[k + 1], 1 / (plev[k] - plev[k + 1]), 0)
    int16_t kguess[kGuessBins];
    float2 sc[3][NSC];     // scales of u, v, omega per level as pairs (slot 0, slot 1)
};
using Smem = SmemT<kMaxNZ>;
// level scales in shared memory only for fp16 pair records (bf16 pair records hold scaled values)
template <int ST> using SmemFor = SmemT<ST == MPTRAC_FP16 ? kMaxNZ : 1>;

// Cell of a point: indices (lon i, lat j, lower level k) and the
// interpolation weights as (f, g = 1 - f) pairs.  All indices are clamped into
// the grid whatever the input.
struct Cell {
    int i, j, k;
    float fx, gx, fy, gy, fz, gz;
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

// Longitude and latitude enter as e = lon - lon0 and d = lat - lat0 in
// float-float, and both cell coordinates x = e / dlon, y = d / dlat are formed
// in float-float: on a fine grid whose spacing has no exact float inverse
// (0.3 degrees), a float32 x near the eastern end (x ~ 1200) would carry
// ~1e-4 cells of error, which steep grid-scale winds turn into metres per
// hour.  Both latitude weights are computed directly, so that next to a pole
// the small weight keeps its relative precision (winds there vanish like the
// distance to the pole while the longitude increment divides by cos(lat)).
// The level search starts from `k_hint` (the level of the previous evaluation;
// < 0: none), else from the ln(p) table, and walks to the bracketing pair.
template <class S>
__device__ __forceinline__ Cell locate(ff e, ff d, float p, const Geo& g, const S& s, int k_hint) {
    Cell c;
    // e is in [0, 360), so xh >= 0 and xh - floor(xh) is exact and in [0, 1);
    // i == nx (xh rounded up to nx) wraps to 0, and the clamp keeps a NaN's
    // index inside the grid.  The correction xe is below an ulp of xh: the
    // weights may leave [0, 1] by that much, a continuous extrapolation.
    const float xh = __fmul_rn(e.hi, g.inv_dlon);
    float xe = fmaf(e.hi, g.inv_dlon, -xh);
    xe = fmaf(e.hi, g.inv_dlon_lo, xe);
    xe = fmaf(e.lo, g.inv_dlon, xe);
    const float xf = floorf(xh);
    int i = (int)xf;
    if (i >= g.nx) i -= g.nx;
    c.i = min(max(i, 0), g.nx - 1);
    c.fx = __fadd_rn(__fsub_rn(xh, xf), xe);
    c.gx = __fsub_rn(1.f, c.fx);

    // y = d / dlat as float-float (yh + ye); the row index is clamped as a
    // float (exact small integers), which saves converting it back
    const float yh = d.hi * g.inv_dlat;
    float ye = fmaf(d.hi, g.inv_dlat, -yh);
    ye = fmaf(d.hi, g.inv_dlat_lo, ye);
    ye = fmaf(d.lo, g.inv_dlat, ye);
    const float jf = fminf(fmaxf(floorf(yh), 0.f), (float)(g.ny - 2));
    c.j = (int)jf;
    c.fy = clamp01(__fadd_rn(__fsub_rn(yh, jf), ye));
    c.gy = clamp01(__fsub_rn(__fsub_rn(jf + 1.f, yh), ye));

    const float pc = fminf(fmaxf(p, g.pmin), g.pmax);
    int k = k_hint;
    if (k < 0) {
        int b = (int)((__logf(pc) - g.lnp_top) * g.inv_dln);
        b = min(max(b, 0), g.nbins - 1);
        k = s.kguess[b];
    }
    // one 16-byte load gives both bounds of level k and the inverse spacing; the
    // walk to another level (rare: the level of the previous evaluation is the
    // first guess) reloads it
    float4 lv = s.lv[k];
    if (k > 0 && lv.x < pc) {
        do { --k; } while (k > 0 && s.plev[k] < pc);
        lv = s.lv[k];
    } else if (k < g.nz - 2 && lv.y >= pc) {
        do { ++k; } while (k < g.nz - 2 && s.plev[k + 1] >= pc);
        lv = s.lv[k];
    }
    c.k = k;
    c.fz = clamp01((lv.x - pc) * lv.z);
    c.gz = 1.f - c.fz;
    return c;
}

struct Wind {
    float u, v, w;
};

// Pairs of float32 values in one 64-bit register, operated on by Blackwell's
// packed float32x2 instructions (each lane rounds exactly like the scalar
// instruction).  Lane s holds met slot s's snapshot, so one instruction
// interpolates both snapshots; the time weights come per lane.
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
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The 8 corners of one cell on both snapshots, (u, v, omega) decoded and
// scaled, kept per particle.  A particle moves about 1/60 of a 1-degree cell
// per step, so consecutive wind evaluations almost always fall into the cell
// already held here and need no global memory access at all: the gather from
// L1/L2 is paid only when the particle changes cell.  Corner order q: bit 0 =
// i+1, bit 1 = j+1, bit 2 = k+1; each value is a pair (snapshot 0, snapshot 1).
//
// RegCache holds the 24 pairs in registers (48 registers per thread).
struct RegCache {
    int col, k;               // cached cell (record index of column (j, i), lower level); col < 0: empty
    f2_t u[8], v[8], w[8];
    static constexpr int kGroups = 1;   // corners fetched in one group of 8
    __device__ __forceinline__ void init(ulonglong2*) { col = -1; k = -1; }
    __device__ __forceinline__ void store(int, const f2_t* U, const f2_t* V, const f2_t* W) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            u[q] = U[q];
            v[q] = V[q];
            w[q] = W[q];
        }
    }
    __device__ __forceinline__ void get(int var, f2_t* x) const {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = var == 0 ? u[q] : (var == 1 ? v[q] : w[q]);
    }
};

// SmemCache holds them in the thread's slice of a block-wide shared array:
// 12 slots of 16 bytes (two corners of one variable), slot e of thread t at
// [e * BLOCK + t], so a warp reads 512 contiguous bytes per slot.  It frees
// the registers for more resident warps at the cost of 12 shared loads per
// wind evaluation.  It is filled one level (4 corners) at a time, which halves
// the records in flight during a fetch.
template <int BLOCK>
struct SmemCache {
    static constexpr int kGroups = 2;
    int col, k;
    ulonglong2* slot;
    __device__ __forceinline__ void init(ulonglong2* base) {
        col = -1;
        k = -1;
        slot = base + threadIdx.x;
    }
    // corners 4 gi .. 4 gi + 3 (U[0..3] etc.)
    __device__ __forceinline__ void store(int gi, const f2_t* U, const f2_t* V, const f2_t* W) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int h = 2 * gi + hh;
            slot[(0 * 4 + h) * BLOCK] = make_ulonglong2(U[2 * hh], U[2 * hh + 1]);
            slot[(1 * 4 + h) * BLOCK] = make_ulonglong2(V[2 * hh], V[2 * hh + 1]);
            slot[(2 * 4 + h) * BLOCK] = make_ulonglong2(W[2 * hh], W[2 * hh + 1]);
        }
    }
    // The empty asm keeps the compiler from hoisting the loads of all three
    // variables to the top of an evaluation (48 registers in flight).
    __device__ __forceinline__ void get(int var, f2_t* x) const {
        asm volatile("" ::: "memory");
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const ulonglong2 t = slot[(var * 4 + h) * BLOCK];
            x[2 * h] = t.x;
            x[2 * h + 1] = t.y;
        }
    }
};

// One interleaved pair record: (u, v, omega, T) x (slot 0, slot 1).
template <int ST> struct PairRecT;
template <> struct PairRecT<MPTRAC_FP32> { static constexpr int kBytes = 32; };
template <> struct PairRecT<MPTRAC_BF16> { static constexpr int kBytes = 16; };
template <> struct PairRecT<MPTRAC_FP16> { static constexpr int kBytes = 16; };

// float32 pair record -> u, v, omega pairs, straight from one 32-byte load
__device__ __forceinline__ void load_pair32(const void* p, f2_t& u, f2_t& v, f2_t& w) {
    f2_t t;
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(u), "=l"(v), "=l"(w), "=l"(t) : "l"(p));
}

// a word of two 16-bit codes (slot 0 low, slot 1 high) -> pair of floats
template <int ST>
__device__ __forceinline__ f2_t decode_pair16(uint32_t x) {
    if (ST == MPTRAC_BF16) return f2_pack(__uint_as_float(x << 16), __uint_as_float(x & 0xFFFF0000u));
    return f2_pack(__half2float(__ushort_as_half((unsigned short)(x & 0xFFFFu))),
                   __half2float(__ushort_as_half((unsigned short)(x >> 16))));
}

template <int ST, class S, class C>
__device__ __forceinline__ void fetch_corners(const MetPair& mp, const S& s, const Geo& g, const Cell& c,
                                              int col, C& cc) {
    const int i1 = (c.i + 1 == g.nx) ? 0 : c.i + 1;
    const int row1 = col - c.i + g.nx;
    const int base[4] = {col * g.nz + c.k, (col - c.i + i1) * g.nz + c.k, (row1 + c.i) * g.nz + c.k,
                         (row1 + i1) * g.nz + c.k};
    const char* rec = static_cast<const char*>(mp.rec);
    constexpr int RB = PairRecT<ST>::kBytes;
    constexpr int QG = 8 / C::kGroups;   // corners per group
#pragma unroll 1
    for (int gi = 0; gi < C::kGroups; ++gi) {
        f2_t U[QG], V[QG], W[QG];
        if (ST == MPTRAC_FP32) {
#pragma unroll
            for (int qq = 0; qq < QG; ++qq) {
                const int q = gi * QG + qq;
                load_pair32(rec + (size_t)(base[q & 3] + (q >> 2)) * RB, U[qq], V[qq], W[qq]);
            }
        } else {
            uint4 r[QG];
#pragma unroll
            for (int qq = 0; qq < QG; ++qq) {
                const int q = gi * QG + qq;
                r[qq] = __ldg(reinterpret_cast<const uint4*>(rec + (size_t)(base[q & 3] + (q >> 2)) * RB));
            }
#pragma unroll
            for (int qq = 0; qq < QG; ++qq) {
                if constexpr (ST == MPTRAC_BF16) {   // bf16 pair records hold the scaled values
                    U[qq] = decode_pair16<ST>(r[qq].x);
                    V[qq] = decode_pair16<ST>(r[qq].y);
                    W[qq] = decode_pair16<ST>(r[qq].z);
                } else {
                    const int k = c.k + ((gi * QG + qq) >> 2);
                    U[qq] = f2_mul(decode_pair16<ST>(r[qq].x), *reinterpret_cast<const f2_t*>(&s.sc[0][k]));
                    V[qq] = f2_mul(decode_pair16<ST>(r[qq].y), *reinterpret_cast<const f2_t*>(&s.sc[1][k]));
                    W[qq] = f2_mul(decode_pair16<ST>(r[qq].z), *reinterpret_cast<const f2_t*>(&s.sc[2][k]));
                }
            }
        }
        cc.store(gi, U, V, W);
    }
    cc.col = col;
    cc.k = c.k;
}

// The 8 trilinear corner weights, each as a pair (same weight for both
// snapshots); corner order as in the corner caches.
struct Weights8 {
    f2_t w[8];
};

__device__ __forceinline__ Weights8 weights8(const Cell& c) {
    // products in scalar form (both lanes of a weight are equal), then paired
    const float a00 = c.gy * c.gz, a10 = c.fy * c.gz, a01 = c.gy * c.fz, a11 = c.fy * c.fz;
    const float w[8] = {c.gx * a00, c.fx * a00, c.gx * a10, c.fx * a10,
                        c.gx * a01, c.fx * a01, c.gx * a11, c.fx * a11};
    Weights8 r;
#pragma unroll
    for (int q = 0; q < 8; ++q) r.w[q] = f2_pack(w[q], w[q]);
    return r;
}

// trilinear interpolation of 8 corner pairs: sum of weight x corner value
__device__ __forceinline__ f2_t trilinear(const f2_t* x, const Weights8& W) {
    f2_t acc = f2_mul(W.w[0], x[0]);
#pragma unroll
    for (int q = 1; q < 8; ++q) acc = f2_fma(W.w[q], x[q], acc);
    return acc;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Interpolated value and subgrid variance of 8 corner pairs (both snapshots
// at once).  The variance is the spread of the corners about the interpolated
// value weighted by the interpolation weights, sum_q w_q (x_q - mean)^2.  With
// the weights summing to 1 it equals S - m^2, where m = sum_q w_q (x_q - x_0)
// and S = sum_q w_q (x_q - x_0)^2 are taken relative to corner 0, and mean =
// x_0 + m; corner 0's weight is not needed.  The rounding of S - m^2 is at
// most a few float32 ulps of S: where the true spread is smaller (a point on
// or within ~1e-7 cells of a corner other than 0) the result can come out
// slightly negative, and the caller clamps it at 0.  The subgrid sigma then
// errs by at most about sqrt(2 eps) |x_q - x_0|, 3.5e-4 of the corner difference.
__device__ __forceinline__ void mean_and_var(const f2_t* x, const Weights8& W, f2_t& mean, f2_t& var) {
    f2_t m, S;
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        const f2_t y = f2_sub(x[q], x[0]);
        const f2_t wy = f2_mul(W.w[q], y);
        if (q == 1) {
            m = wy;
            S = f2_mul(wy, y);
        } else {
            m = f2_add(m, wy);
            S = f2_fma(wy, y, S);
        }
    }
    mean = f2_add(x[0], m);
    var = f2_fma(m ^ 0x8000000080000000ull, m, S);   // S - m^2 (sign bits of both lanes flipped)
}

// linear interpolation in time of a (slot 0, slot 1) pair with the lane
// weights (wl, wh): 1 - w for the earlier snapshot's lane, w for the later's
__device__ __forceinline__ float tlerp(f2_t ab, float wl, float wh) {
    float a, b;
    f2_split(ab, a, b);
    return fmaf(wh, b, wl * a);
}

// Wind at a located point and lane time weights (wl, wh), with the subgrid
// variances when SIG.
template <int ST, bool SIG, class S, class C>
__device__ __forceinline__ void eval_wind(const MetPair& mp, const S& s, const Geo& g, const Cell& c,
                                          float wl, float wh, C& cc, Wind& out, Wind& var) {
    const int col = c.j * g.nx + c.i;
    if (col != cc.col || c.k != cc.k) fetch_corners<ST>(mp, s, g, c, col, cc);
    const Weights8 W = weights8(c);
    float o[3], sg[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        f2_t x[8];
        cc.get(v, x);
        if (SIG) {
            f2_t t, vr;
            mean_and_var(x, W, t, vr);
            o[v] = tlerp(t, wl, wh);
            sg[v] = fmaxf(tlerp(vr, wl, wh), 0.f);   // rounding of S - m^2 below 0 (see mean_and_var)
        } else {
            o[v] = tlerp(trilinear(x, W), wl, wh);
        }
    }
    out = Wind{o[0], o[1], o[2]};
    if (SIG) var = Wind{sg[0], sg[1], sg[2]};
}

// sc0 / sc1: scales of slot 0 / 1 (read only when `scales`)
template <int NSC>
__device__ __forceinline__ void load_tables(SmemT<NSC>& s, const Geo& g, const float* sc0, const float* sc1,
                                            bool scales) {
    for (int q = threadIdx.x; q < g.nz; q += blockDim.x) {
        s.plev[q] = g.plev[q];
        s.lv[q] = make_float4(g.plev[q], q + 1 < g.nz ? g.plev[q + 1] : g.plev[q], g.inv_dp[q], 0.f);
    }
    for (int q = threadIdx.x; q < g.nbins; q += blockDim.x) s.kguess[q] = g.kguess[q];
    if (NSC > 1 && scales) {
        for (int q = threadIdx.x; q < 3 * g.nz; q += blockDim.x) {
            const int var = q / g.nz, k = q - var * g.nz;
            s.sc[var][k] = make_float2(sc0[var * g.nz + k], sc1[var * g.nz + k]);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Pieces of the step: midpoint position rules, random draws
// ---------------------------------------------------------------------------
// Midpoint position rules: latitude reflected over the poles (longitude +
// 180), longitude wrapped into [0, 360) (as e = lon - lon0).  The pressure
// needs no rule here: `locate` clamps it to the level range.
__device__ __forceinline__ void midpoint_bc(ff& e, ff& d, const Geo& g) {
    if (!(d.hi < g.dn && d.hi > g.ds && e.hi < 360.f && e.hi >= 0.f)) horizontal_rules(e, d, g);
}

// sqrt(x), x >= 0 (a weighted sum of squares), by the approximate square root
// instruction.  Written as PTX so that every instantiation runs the same
// instruction: results must not depend on the launch variant.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Gaussian draws of one step from counters (id, step, 0, release) and
// (id, step, 1, release): their normals are used in order, turbulence taking
// the first three of draw 0, mesoscale the fourth of draw 0 and the first two
// of draw 1 -- three Box-Muller pairs per step.
struct Normals {
    float t0, t1, t2;   // turbulence: east, north, vertical
    float m0, m1, m2;   // mesoscale: u, v, omega
};

// Round-0 words of a particle's counters (see philox_after_round0).
struct Round0 {
    uint32_t z, w;
};
__device__ __forceinline__ Round0 round0(const StepArgs& a, uint32_t pid, uint32_t rel) {
    uint32_t hi, lo;
    mul_wide(0xD2511F53u, pid, hi, lo);
    return {hi ^ rel ^ a.ks[1], lo};
}

// draw 0: the turbulent normals and the first mesoscale one
__device__ __forceinline__ void draw_turb(const StepArgs& a, Round0 r0, uint32_t step, Normals& z) {
    const uint4 wd = philox_after_round0(step, 0u, r0.z, r0.w, a.ks);
    box_muller(wd.x, wd.y, z.t0, z.t1);
    box_muller(wd.z, wd.w, z.t2, z.m0);
}
// draw 1: the other two mesoscale normals
__device__ __forceinline__ void draw_meso(const StepArgs& a, Round0 r0, uint32_t step, Normals& z) {
    const uint4 wd = philox_after_round0(step, 1u, r0.z, r0.w, a.ks);
    box_muller(wd.x, wd.y, z.m1, z.m2);
}

// Hand-off of one particle to the sort that follows the launch: its final
// state goes to the workspace copies (the mesoscale perturbations already
// there when `meso_done`), its cell key to keys[idx], and the key's lowest
// digit to the histogram of its 1024-particle tile.  Lanes of a warp with the
// same digit add their count with one atomic.
template <class S>
__device__ __forceinline__ void hand_off(const StepArgs& a, const S& s, int64_t idx, double lon, double lat,
                                         double p, uint32_t pid, bool meso_done) {
    const SortEmit& e = a.emit;
    e.copy.d[0][idx] = lon;
    e.copy.d[1][idx] = lat;
    e.copy.d[2][idx] = p;
    e.copy.u[0][idx] = pid;
    if (e.copy.u[1]) e.copy.u[1][idx] = a.release[idx];
    if (!meso_done) {
        const float* src[3] = {a.up, a.vp, a.wp};
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (e.copy.f[c]) e.copy.f[c][idx] = src[c][idx];
    }
    const uint32_t key = cell_key(lon, lat, p, a.geo, s.plev, s.kguess, a.geo.plev_d);
    e.keys[idx] = key;
    const uint32_t digit = key & (kSortRadix - 1);
    const unsigned peers = __match_any_sync(__activemask(), digit);
    if ((__ffs(peers) - 1) == (int)(threadIdx.x & 31))
        atomicAdd(&e.hist[(int64_t)digit * e.ntiles + idx / kSortTileKeys], (uint32_t)__popc(peers));
}

// ---------------------------------------------------------------------------
// The particle kernel
// ---------------------------------------------------------------------------
// CACHE: 0 = corner cache in registers, 1 = in shared memory.
template <int ST, int MODE, int BLOCK, int MINB, int CACHE>
__global__ void __launch_bounds__(BLOCK, MINB) k_transport(const __grid_constant__ StepArgs a) {
    __shared__ SmemFor<ST> s;
    __shared__ ulonglong2 s_cc[CACHE ? 12 * BLOCK : 1];
    using Cache = typename std::conditional<CACHE != 0, SmemCache<BLOCK>, RegCache>::type;
    load_tables(s, a.geo, a.mp.scales[0], a.mp.scales[1], ST == MPTRAC_FP16);
    const Geo& g = a.geo;
    constexpr bool FULL = (MODE == MODE_STEP_FULL);
    constexpr bool ADVECT = (MODE != MODE_DIFFUSE);
    // draws made first (see below) only where the registers allow it (the
    // 128-register variants)
    constexpr bool EARLY_DRAWS = FULL && CACHE == 0 && MINB * BLOCK <= 512;
    const bool use_meso = FULL || ((MODE != MODE_ADVECT) && a.meso);
    const bool use_turb = FULL || ((MODE != MODE_ADVECT) && a.turb);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n; idx += stride) {
        const bool masked = a.mask && !a.mask[idx];
        int nlo = 0, nhi = a.nsteps;
        uint32_t rel = 0;
        if (!masked && a.release) {
            rel = a.release[idx];
            if (a.win) {
                if (rel < (uint32_t)a.n_rel) {
                    const int2 wv = a.win[rel];
                    nlo = wv.x;
                    nhi = wv.y;
                } else {
                    nlo = nhi = 0;
                }
            }
        }
        const bool emit = a.emit.keys != nullptr;
        if (masked || nlo >= nhi) {   // left as it is
            if (emit) hand_off(a, s, idx, a.lon[idx], a.lat[idx], a.p[idx], a.id[idx], false);
            continue;
        }
        ff lon = ff_make(a.lon[idx] - g.lon0_d);   // longitude as e = lon - lon0
        ff d = ff_make(a.lat[idx] - g.lat0_d);     // latitude as d = lat - lat0
        ff p = ff_make(a.p[idx]);
        const uint32_t pid = a.id[idx];
        const Round0 r0 = round0(a, pid, rel);
        float up = 0.f, vp = 0.f, wp = 0.f;
        Cache cc;
        cc.init(s_cc);
        if (use_meso) {
            up = a.up[idx];
            vp = a.vp[idx];
            wp = a.wp[idx];
        }
        for (int sidx = nlo; sidx < nhi; ++sidx) {
            const uint32_t step = (uint32_t)(a.step0 + (uint64_t)sidx);
            Normals z{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            // The draws do not depend on the position: with both diffusion
            // parts compiled in they are made first, so that their integer
            // work interleaves with the dependent chain of the advection.
            if (EARLY_DRAWS) {
                draw_turb(a, r0, step, z);
                draw_meso(a, r0, step, z);
            }
            // increments of this step (lon and lat in degrees, p in Pa)
            float ilon = 0.f, ilat = 0.f, ip = 0.f;
            Wind var{0.f, 0.f, 0.f};
            if (ADVECT) {
                // ---- module_advection: explicit midpoint ----
                const float wl0 = a.wt[4 * sidx], wh0 = a.wt[4 * sidx + 1];
                const float wlm = a.wt[4 * sidx + 2], whm = a.wt[4 * sidx + 3];
                const Cell c1 = locate(lon, d, p.hi, g, s, cc.k);
                Wind V;
                if (MODE != MODE_ADVECT && use_meso)
                    eval_wind<ST, true>(a.mp, s, g, c1, wl0, wh0, cc, V, var);
                else
                    eval_wind<ST, false>(a.mp, s, g, c1, wl0, wh0, cc, V, var);
                const float cl = coslat(d, 0.f, g);
                ff lon_m = ff_add_inc_raw(lon, __fdividef(a.hk * V.u, cl));
                ff d_m = ff_add_inc(d, a.hk * V.v);
                const float p_m = p.hi + a.half_dt * V.w;
                midpoint_bc(lon_m, d_m, g);
                const Cell c2 = locate(lon_m, d_m, p_m, g, s, cc.k);
                Wind V2, dummy;
                eval_wind<ST, false>(a.mp, s, g, c2, wlm, whm, cc, V2, dummy);
                const float cl2 = coslat(d_m, 0.f, g);
                ilon = __fdividef(a.dk * V2.u, cl2);
                ilat = a.dk * V2.v;
                ip = a.dt * V2.w;
            } else if (use_meso) {
                const Cell c1 = locate(lon, d, p.hi, g, s, cc.k);
                Wind V;
                eval_wind<ST, true>(a.mp, s, g, c1, a.wt[4 * sidx], a.wt[4 * sidx + 1], cc, V, var);
            }
            if (MODE != MODE_ADVECT && (use_turb || use_meso)) {
                // ---- module_diffusion_turb / module_diffusion_meso ----
                // at the position after advection: lat + ilat, p + ip
                if (!EARLY_DRAWS && (use_turb || use_meso)) draw_turb(a, r0, step, z);
                if (!EARLY_DRAWS && use_meso) draw_meso(a, r0, step, z);
                float dxm = 0.f, dym = 0.f, dpp = 0.f;
                if (use_turb) {
                    dxm = a.sh * z.t0;
                    dym = a.sh * z.t1;
                    dpp = -(p.hi + ip) * (a.sv * z.t2) * a.inv_H;
                }
                if (use_meso) {
                    up = fmaf(a.r_ar, up, a.a_ar * sqrt_approx(var.u) * z.m0);
                    vp = fmaf(a.r_ar, vp, a.a_ar * sqrt_approx(var.v) * z.m1);
                    wp = fmaf(a.r_ar, wp, a.a_ar * sqrt_approx(var.w) * z.m2);
                    dxm += up * a.dt;
                    dym += vp * a.dt;
                    dpp += wp * a.dt;
                }
                const float c3 = coslat(d, ilat, g);
                ilon += __fdividef(dxm * a.kdeg, c3);
                ilat += dym * a.kdeg;
                ip += dpp;
            }
            lon = ff_add_inc(lon, ilon);
            d = ff_add_inc(d, ilat);
            p = ff_add_inc(p, ip);
            // ---- module_position ----
            position_bc(lon, d, p, g);
        }
        const double lon_out = ff_val(lon) + g.lon0_d, lat_out = ff_val(d) + g.lat0_d, p_out = ff_val(p);
        if (emit) {
            if (use_meso) {
                a.emit.copy.f[0][idx] = up;
                a.emit.copy.f[1][idx] = vp;
                a.emit.copy.f[2][idx] = wp;
            }
            hand_off(a, s, idx, lon_out, lat_out, p_out, pid, use_meso);
        } else {
            a.lon[idx] = lon_out;
            a.lat[idx] = lat_out;
            a.p[idx] = p_out;
            if (use_meso) {
                a.up[idx] = up;
                a.vp[idx] = vp;
                a.wp[idx] = wp;
            }
        }
    }
}

// Release windows: for each release the contiguous range [lo, hi) of local
// steps (n_begin + n) whose time t + (n_begin + n) dt lies in [t_start, t_end).  Same float64
// expression as the host-side definition (no fused multiply-add).
__global__ void k_windows(const double* ts, const double* te, int nrel, double t, double dt,
                          int n_begin, int nsteps, int2* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrel) return;
    const double a = ts[r], b = te[r];
    int lo = -1, hi = -1;
    for (int n = 0; n < nsteps; ++n) {
        const double tn = __dadd_rn(t, __dmul_rn((double)(n_begin + n), dt));
        if (tn >= a && tn < b) {
            if (lo < 0) lo = n;
            hi = n + 1;
        }
    }
    out[r] = (lo < 0) ? make_int2(0, 0) : make_int2(lo, hi);
}

template <int ST>
__global__ void __launch_bounds__(kBlock) k_interp(Geo g, MetPair mp, float wl, float wh,
                                                   int64_t n, const double* lon,
                                                   const double* lat, const double* p,
                                                   float* ou, float* ov, float* ow,
                                                   float* ovar) {
    __shared__ Smem s;
    load_tables(s, g, mp.scales[0], mp.scales[1], ST == MPTRAC_FP16);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const Cell c = locate(ff_make(lon[idx] - g.lon0_d), ff_make(lat[idx] - g.lat0_d), ff_make(p[idx]).hi, g, s, -1);
        Wind V, var;
        RegCache cc;
        cc.init(nullptr);
        eval_wind<ST, true>(mp, s, g, c, wl, wh, cc, V, var);
        ou[idx] = V.u;
        ov[idx] = V.v;
        ow[idx] = V.w;
        if (ovar) {
            ovar[idx] = var.u;
            ovar[n + idx] = var.v;
            ovar[2 * n + idx] = var.w;
        }
    }
}

// module_meteo: u, v, omega, T at the particle positions (4D linear, float32)
template <int ST>
__global__ void __launch_bounds__(kBlock) k_sample(Geo g, MetView m0, MetView m1, float w, int64_t n,
                                                   const double* lon, const double* lat, const double* p,
                                                   float* out) {
    __shared__ Smem s;
    load_tables(s, g, nullptr, nullptr, false);
    using R = typename RecT<ST>::T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const Cell c = locate(ff_make(lon[idx] - g.lon0_d), ff_make(lat[idx] - g.lat0_d), ff_make(p[idx]).hi, g, s, -1);
        const int i1 = (c.i + 1 == g.nx) ? 0 : c.i + 1;
        const int col[4] = {c.j * g.nx + c.i, c.j * g.nx + i1, (c.j + 1) * g.nx + c.i, (c.j + 1) * g.nx + i1};
        float res[2][4];
#pragma unroll   // the 16 record loads of both snapshots in flight together
        for (int t = 0; t < 2; ++t) {
            const R* rec = static_cast<const R*>(t ? m1.rec : m0.rec);
            const float* sc = t ? m1.scales : m0.scales;
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[q] = decode<ST>(__ldg(rec + col[q & 3] * g.nz + c.k + (q >> 2)));
                if (ST != MPTRAC_FP32) {
                    const int k = c.k + (q >> 2);
                    v[q].x *= sc[k];
                    v[q].y *= sc[g.nz + k];
                    v[q].z *= sc[2 * g.nz + k];
                    v[q].w *= sc[3 * g.nz + k];
                }
            }
#define MPTRAC_TRI4(comp, dst)                                                             \
    {                                                                                      \
        const float e0 = fmaf(v[1].comp, c.fx, v[0].comp * c.gx);                          \
        const float e1 = fmaf(v[3].comp, c.fx, v[2].comp * c.gx);                          \
        const float e2 = fmaf(v[5].comp, c.fx, v[4].comp * c.gx);                          \
        const float e3 = fmaf(v[7].comp, c.fx, v[6].comp * c.gx);                          \
        dst = fmaf(fmaf(e3, c.fy, e2 * c.gy), c.fz, fmaf(e1, c.fy, e0 * c.gy) * c.gz);    \
    }
            MPTRAC_TRI4(x, res[t][0])
            MPTRAC_TRI4(y, res[t][1])
            MPTRAC_TRI4(z, res[t][2])
            MPTRAC_TRI4(w, res[t][3])
#undef MPTRAC_TRI4
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) out[v * n + idx] = fmaf(w, res[1][v] - res[0][v], res[0][v]);
    }
}

// module_sedi: Stokes settling with the Cunningham slip correction, T from the
// met snapshots (4D linear), dp = rho_air g v_s dt per step, p clamped.
struct SediArgs {
    Geo g;
    MetView m0, m1;
    int64_t n;
    const double *lon, *lat;
    double* p;
    const float *radius, *rho_p;
    int nsteps;
    float dt, w0, dw;
};

template <int ST>
__global__ void __launch_bounds__(kBlock) k_sedi(const SediArgs a) {
    __shared__ Smem s;
    load_tables(s, a.g, nullptr, nullptr, false);
    const Geo& g = a.g;
    using R = typename RecT<ST>::T;
    constexpr float Rd = 287.058f, G = 9.80665f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n; idx += stride) {
        const ff e = ff_make(a.lon[idx] - g.lon0_d);
        const ff d = ff_make(a.lat[idx] - g.lat0_d);
        ff p = ff_make(a.p[idx]);
        const float r = a.radius[idx], rp = a.rho_p[idx];
        int ccol = -1, ck = -1;
        float T0[8], T1[8];
        for (int n = 0; n < a.nsteps; ++n) {
            const Cell c = locate(e, d, p.hi, g, s, ck);
            const int col = c.j * g.nx + c.i;
            if (col != ccol || c.k != ck) {
                const int i1 = (c.i + 1 == g.nx) ? 0 : c.i + 1;
                const int cols[4] = {col, col - c.i + i1, col + g.nx, col + g.nx - c.i + i1};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = c.k + (q >> 2);
                    const int64_t o = (int64_t)cols[q & 3] * g.nz + k;
                    T0[q] = decode<ST>(__ldg(static_cast<const R*>(a.m0.rec) + o)).w;
                    T1[q] = decode<ST>(__ldg(static_cast<const R*>(a.m1.rec) + o)).w;
                    if (ST != MPTRAC_FP32) {
                        T0[q] *= a.m0.scales[3 * g.nz + k];
                        T1[q] *= a.m1.scales[3 * g.nz + k];
                    }
                }
                ccol = col;
                ck = c.k;
            }
            float tr[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const float* v = t ? T1 : T0;
                const float e0 = fmaf(v[1], c.fx, v[0] * c.gx), e1 = fmaf(v[3], c.fx, v[2] * c.gx);
                const float e2 = fmaf(v[5], c.fx, v[4] * c.gx), e3 = fmaf(v[7], c.fx, v[6] * c.gx);
                tr[t] = fmaf(fmaf(e3, c.fy, e2 * c.gy), c.fz, fmaf(e1, c.fy, e0 * c.gy) * c.gz);
            }
            const float w = a.w0 + (float)n * a.dw;
            const float T = fmaf(w, tr[1] - tr[0], tr[0]);
            const float rho = p.hi / (Rd * T);
            const float tt = T * (1.0f / 296.16f);
            const float eta = 1.8325e-5f * (416.16f / (T + 120.0f)) * tt * sqrtf(tt);
            const float vbar = sqrtf(8.0f * Rd * T * 0.31830988618379067f);
            const float kn = 2.0f * eta / (rho * vbar) / r;
            const float cc = 1.0f + kn * (1.257f + 0.4f * expf(-1.1f / kn));
            const float vs = 2.0f * r * r * (rp - rho) * G * cc / (9.0f * eta);
            p = ff_add(p, rho * G * vs * a.dt);
            if (ff_less(p, g.pmin, g.pmin_lo)) { p.hi = g.pmin; p.lo = g.pmin_lo; }
            if (ff_greater(p, g.pmax, g.pmax_lo)) { p.hi = g.pmax; p.lo = g.pmax_lo; }
        }
        a.p[idx] = ff_val(p);
    }
}

__global__ void k_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1,
                         uint32_t* out, float* normals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 c = make_uint4(ctr[i], ctr[n + i], ctr[2 * n + i], ctr[3 * n + i]);
        const uint4 wd = philox4x32_10(c, k0, k1);
        out[i] = wd.x;
        out[n + i] = wd.y;
        out[2 * n + i] = wd.z;
        out[3 * n + i] = wd.w;
        if (normals) {
            float z0, z1, z2, z3;
            box_muller(wd.x, wd.y, z0, z1);
            box_muller(wd.z, wd.w, z2, z3);
            normals[i] = z0;
            normals[n + i] = z1;
            normals[2 * n + i] = z2;
            normals[3 * n + i] = z3;
        }
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (int)b;
}

// Launch variants of the fused step (threads per block, minimum resident blocks
// per SM -- which caps the registers -- and where the corner cache lives):
// 0 = (256, 2) 128 registers, 1 = (128, 4) 128 registers in finer blocks,
// 2 = (128, 5) 96 registers, 20 warps per SM; 3 = (128, 6) corner cache in
// shared memory, 80 registers, 24 warps per SM; 4 = (128, 7) the same with 72
// registers, 28 warps per SM (24 with 16-bit storage, whose scale tables take
// shared memory too); 5 = (64, 10) 96 registers in the smallest blocks; 6 =
// (512, 1) 128 registers in the largest.
template <int ST, int MODE, int BLOCK, int MINB, int CACHE>
cudaError_t launch_step_variant(const StepArgs& a, int grid, int schedule, cudaStream_t s) {
    auto kern = k_transport<ST, MODE, BLOCK, MINB, CACHE>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        dev = 0;
    }
    if (CACHE) {
        // prefer the largest shared-memory carveout (a per-device function attribute)
        static std::atomic<int> carveout_set[kMaxDevices];
        if (!carveout_set[dev].load(std::memory_order_relaxed)) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                (void)cudaGetLastError();
            carveout_set[dev].store(1, std::memory_order_relaxed);
        }
    }
    if (schedule == 1) {
        // resident blocks per SM of this instantiation, per device
        static std::atomic<int> per_sm_cache[kMaxDevices];
        int per_sm = per_sm_cache[dev].load(std::memory_order_relaxed);
        if (per_sm <= 0) {
            int v = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, BLOCK, 0) != cudaSuccess) {
                (void)cudaGetLastError();
                v = MINB;
            }
            per_sm = v;
            per_sm_cache[dev].store(v, std::memory_order_relaxed);
        }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t need = (a.n + BLOCK - 1) / BLOCK;
        grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), need));
    } else {
        // schedule k >= 2: k particles per thread (the kernel's loop strides over the grid)
        const int64_t per_block = (int64_t)BLOCK * (schedule >= 2 ? schedule : 1);
        grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + per_block - 1) / per_block, (int64_t)1 << 20));
    }
    kern<<<grid, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_transport_st(int mode, const StepArgs& a, int grid, int variant, int schedule,
                                cudaStream_t s) {
    if (mode == MODE_STEP && a.turb && a.meso) {
        switch (variant) {
            case 1: return launch_step_variant<ST, MODE_STEP_FULL, 128, 4, 0>(a, grid, schedule, s);
            case 2: return launch_step_variant<ST, MODE_STEP_FULL, 128, 5, 0>(a, grid, schedule, s);
            case 3: return launch_step_variant<ST, MODE_STEP_FULL, 128, 6, 1>(a, grid, schedule, s);
            case 4: return launch_step_variant<ST, MODE_STEP_FULL, 128, 7, 1>(a, grid, schedule, s);
            case 5: return launch_step_variant<ST, MODE_STEP_FULL, 64, 10, 0>(a, grid, schedule, s);
            case 6: return launch_step_variant<ST, MODE_STEP_FULL, 512, 1, 0>(a, grid, schedule, s);
            default: return launch_step_variant<ST, MODE_STEP_FULL, kBlock, 2, 0>(a, grid, schedule, s);
        }
    }
    if (mode == MODE_STEP) {
        switch (variant) {
            case 1: return launch_step_variant<ST, MODE_STEP, 128, 4, 0>(a, grid, schedule, s);
            case 2: return launch_step_variant<ST, MODE_STEP, 128, 5, 0>(a, grid, schedule, s);
            case 3: return launch_step_variant<ST, MODE_STEP, 128, 6, 1>(a, grid, schedule, s);
            case 4: return launch_step_variant<ST, MODE_STEP, 128, 7, 1>(a, grid, schedule, s);
            case 5: return launch_step_variant<ST, MODE_STEP, 64, 10, 0>(a, grid, schedule, s);
            case 6: return launch_step_variant<ST, MODE_STEP, 512, 1, 0>(a, grid, schedule, s);
            default: return launch_step_variant<ST, MODE_STEP, kBlock, 2, 0>(a, grid, schedule, s);
        }
    }
    switch (mode) {
        case MODE_ADVECT: k_transport<ST, MODE_ADVECT, kBlock, 2, 0><<<grid, kBlock, 0, s>>>(a); break;
        default: k_transport<ST, MODE_DIFFUSE, kBlock, 2, 0><<<grid, kBlock, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transport(int storage, int mode, const StepArgs& a, int grid, int variant,
                             int schedule, cudaStream_t s) {
    if (grid <= 0) grid = grid_for(a.n);
    note_launches(1);
    switch (storage) {
        case MPTRAC_FP32: return launch_transport_st<MPTRAC_FP32>(mode, a, grid, variant, schedule, s);
        case MPTRAC_BF16: return launch_transport_st<MPTRAC_BF16>(mode, a, grid, variant, schedule, s);
        default: return launch_transport_st<MPTRAC_FP16>(mode, a, grid, variant, schedule, s);
    }
}

cudaError_t launch_windows(const double* ts, const double* te, int nrel, double t, double dt,
                           int n_begin, int nsteps, int2* out, cudaStream_t s) {
    note_launches(1);
    k_windows<<<(nrel + 127) / 128, 128, 0, s>>>(ts, te, nrel, t, dt, n_begin, nsteps, out);
    return cudaGetLastError();
}

cudaError_t launch_interp(int storage, const Geo& g, MetPair mp, float w_lane0, float w_lane1, int64_t n,
                          const double* lon, const double* lat, const double* p, float* ou,
                          float* ov, float* ow, float* ovar, cudaStream_t s) {
    const int grid = strided_grid(n, kBlock, 8);
    note_launches(1);
    switch (storage) {
        case MPTRAC_FP32:
            k_interp<MPTRAC_FP32><<<grid, kBlock, 0, s>>>(g, mp, w_lane0, w_lane1, n, lon, lat, p, ou, ov, ow, ovar);
            break;
        case MPTRAC_BF16:
            k_interp<MPTRAC_BF16><<<grid, kBlock, 0, s>>>(g, mp, w_lane0, w_lane1, n, lon, lat, p, ou, ov, ow, ovar);
            break;
        default:
            k_interp<MPTRAC_FP16><<<grid, kBlock, 0, s>>>(g, mp, w_lane0, w_lane1, n, lon, lat, p, ou, ov, ow, ovar);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sample(int storage, const Geo& g, MetView m0, MetView m1, float w, int64_t n,
                          const double* lon, const double* lat, const double* p, float* out, cudaStream_t s) {
    const int grid = strided_grid(n, kBlock, 8);
    note_launches(1);
    switch (storage) {
        case MPTRAC_FP32: k_sample<MPTRAC_FP32><<<grid, kBlock, 0, s>>>(g, m0, m1, w, n, lon, lat, p, out); break;
        case MPTRAC_BF16: k_sample<MPTRAC_BF16><<<grid, kBlock, 0, s>>>(g, m0, m1, w, n, lon, lat, p, out); break;
        default: k_sample<MPTRAC_FP16><<<grid, kBlock, 0, s>>>(g, m0, m1, w, n, lon, lat, p, out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sedi(int storage, const Geo& g, MetView m0, MetView m1, int64_t n, const double* lon,
                        const double* lat, double* p, const float* radius, const float* rho_p, int nsteps,
                        float dt, float w0, float dw, cudaStream_t s) {
    SediArgs a{g, m0, m1, n, lon, lat, p, radius, rho_p, nsteps, dt, w0, dw};
    const int grid = grid_for(n);   // 20 steps a thread: one particle per thread balances best
    note_launches(1);
    switch (storage) {
        case MPTRAC_FP32: k_sedi<MPTRAC_FP32><<<grid, kBlock, 0, s>>>(a); break;
        case MPTRAC_BF16: k_sedi<MPTRAC_BF16><<<grid, kBlock, 0, s>>>(a); break;
        default: k_sedi<MPTRAC_FP16><<<grid, kBlock, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out,
                          float* normals, cudaStream_t s) {
    note_launches(1);
    k_philox<<<grid_for(n), kBlock, 0, s>>>(ctr, n, k0, k1, out, normals);
    return cudaGetLastError();
}

}  // namespace mptrac
