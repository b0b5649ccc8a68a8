// Cell keys of the particle sort, shared by the sort kernels and by the fused
// step when it hands its results to the sort (arxiv 2211.12616, Section 6:
// particles sorted by the met cell they are in).  key = (j*nx + i)*nz + k.
#pragma once

#include "internal.h"

namespace mptrac {
namespace {

constexpr int kSortTileKeys = 1024;   // keys per histogram tile of the radix sort
constexpr int kSortRadix = 256;       // 8-bit digits

// Cell key from float64 positions, the definition: x = ((lon - lon0) mod 360)
// / dlon, i = floor(x) mod nx; j = floor((lat - lat0) / dlat) clamped to
// [0, ny-2]; k = (number of levels >= clamp(p)) - 1 clamped to [0, nz-2].
// plevd: the float64 levels (a shared-memory copy).  The mod 360 and mod nx
// are skipped where they are the identity (or one subtraction).
__device__ __noinline__ uint32_t cell_key_f64(double lon, double lat, double p, const Geo& g,
                                              const double* plevd) {
    double r = __dsub_rn(lon, g.lon0_d);
    if (!(r >= 0.0 && r < 360.0)) {
        r = fmod(r, 360.0);
        if (r < 0.0) r = __dadd_rn(r, 360.0);
    }
    const double x = __ddiv_rn(r, g.dlon_d);
    long long i = (long long)floor(x);
    if (i >= g.nx) i = (i - g.nx < g.nx) ? i - g.nx : i % g.nx;
    if (i < 0) i = 0;   // x >= 0 here; guards a NaN longitude
    const double y = __ddiv_rn(__dsub_rn(lat, g.lat0_d), g.dlat_d);
    long long j = (long long)floor(y);
    j = j < 0 ? 0 : (j > g.ny - 2 ? g.ny - 2 : j);
    const double pc = fmin(fmax(p, g.pmin_d), g.pmax_d);
    int lo = 0, hi = g.nz;   // plev decreasing: length of the prefix with plev >= pc
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (plevd[mid] >= pc) lo = mid + 1; else hi = mid;
    }
    int k = lo - 1;
    k = k < 0 ? 0 : (k > g.nz - 2 ? g.nz - 2 : k);
    return (uint32_t)((j * g.nx + i) * g.nz + k);
}

struct KeyTables {
    double plev_d[kMaxNZ];
    float plev[kMaxNZ];
    int16_t kguess[kGuessBins];
};

__device__ __forceinline__ void load_key_tables(KeyTables& t, const Geo& g) {
    for (int q = threadIdx.x; q < g.nz; q += blockDim.x) {
        t.plev_d[q] = g.plev_d[q];
        t.plev[q] = g.plev[q];
    }
    for (int q = threadIdx.x; q < g.nbins; q += blockDim.x) t.kguess[q] = g.kguess[q];
}

// float32 of a float64 by truncating its mantissa, with integer operations
// only (|error| < 2^-23 |x|), where the result is a normal float32; zero and
// anything else take the conversion instruction (on the float64 pipe, which
// is narrow on this GPU).
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7FFu;   // float64 biased exponent
    if (e - 897u < 254u) {                     // float32 biased exponent e - 896 in [1, 254]
        const uint32_t mag = (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29);
        return __uint_as_float((hi & 0x80000000u) | mag);
    }
    return (float)x;
}

// Same key, computed in float32 when that is provably identical: the float32
// cell coordinates are within key_mx / key_my cells of the float64 ones (a
// bound derived from the grid on the host, with a factor 2 to spare) and the
// float32 differences p - plev[k] within 1.8e-7 p of the float64 ones, so
// estimates farther than that from every cell face (and p farther than 1e-6
// relative from its bracketing levels) have the same floor / level count as
// the float64 definition.  Anything closer to a face, or outside the regular
// range, takes the float64 path.
// plev / kguess: the float level and first-guess tables (shared-memory
// copies), plevd: the float64 levels.
__device__ __forceinline__ uint32_t cell_key(double lon, double lat, double p, const Geo& g,
                                             const float* plev, const int16_t* kguess, const double* plevd) {
    const float lf = f64_to_f32_trunc(lon), af = f64_to_f32_trunc(lat), pf = f64_to_f32_trunc(p);
    const float x = (lf - g.lon0) * g.inv_dlon;
    const float y = (af - g.lat0) * g.inv_dlat;
    const float xf = floorf(x), yf = floorf(y);
    const float fx = x - xf, fy = y - yf;
    const float mx = g.key_mx, my = g.key_my;
    bool ok = mx < 0.25f && my < 0.25f && (x > mx) && (x < (float)g.nx - mx) && fx > mx && fx < 1.f - mx;
    int j = (int)yf;
    if (y < -my) j = 0;                                          // clamped from below whatever the rounding
    else if (y > (float)(g.ny - 2) + my && y < 1e30f) j = g.ny - 2;  // top cell (clamped)
    else ok = ok && fy > my && fy < 1.f - my && j >= 0 && j <= g.ny - 2;
    // level: first guess from the ln(p) table, refined in float32, accepted
    // only when p is clear of both bracketing levels
    const float pc = fminf(fmaxf(pf, g.pmin), g.pmax);
    int b = (int)((__logf(pc) - g.lnp_top) * g.inv_dln);
    b = min(max(b, 0), g.nbins - 1);
    int k = kguess[b];
    while (k > 0 && plev[k] < pc) --k;
    while (k < g.nz - 2 && plev[k + 1] >= pc) ++k;
    const bool below_top = pf > g.pmax * (1.f + 1e-5f);     // clamps to level 0
    const bool above_bot = pf < g.pmin * (1.f - 1e-5f);     // clamps to the top level
    if (!below_top && !above_bot) {
        const float margin = 1e-6f * pc;
        ok = ok && (plev[k] - pc > margin || k == 0) && (pc - plev[k + 1] > margin || k == g.nz - 2);
        if (k == 0 && !(pc < plev[0] - margin)) ok = false;
        if (k == g.nz - 2 && !(pc > plev[g.nz - 1] + margin)) ok = false;
    }
    if (!ok || !(lf == lf) || !(af == af) || !(pf == pf)) return cell_key_f64(lon, lat, p, g, plevd);
    const int i = (int)xf;
    return (uint32_t)((j * g.nx + i) * g.nz + k);
}

}  // namespace
}  // namespace mptrac
