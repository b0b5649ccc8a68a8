// Internal declarations shared by the translation units of libmptrac.
// Nothing here crosses the C ABI; see include/mptrac.h for the public calls.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "../../include/mptrac.h"

namespace mptrac {

constexpr int kMaxNZ = MPTRAC_MAX_NZ;
constexpr int kMaxStepsPerLaunch = 128;   // time-weight table carried in the kernel parameters
constexpr int kGuessBins = 1024;          // ln(p) bins of the level first-guess table
constexpr int kBlock = 256;               // threads per block of the particle kernels

// Grid geometry as the kernels see it.
struct Geo {
    int nx, ny, nz, nbins;
    float lon0, inv_dlon, lat0, inv_dlat, inv_dlat_lo;   // 1/dlat as float-float (hi, lo)
    float inv_dlon_lo;            // 1/dlon = inv_dlon + inv_dlon_lo (float-float)
    // The particle kernels carry latitude as d = lat - lat0.  The poles and the
    // equator in that coordinate: dn = 90 - lat0, ds = -90 - lat0 as float-float,
    // dmid = -lat0 (exact).
    float dn, dn_lo, ds, ds_lo, dmid;
    float pmin, pmax;             // level range (float)
    float pmin_lo, pmax_lo;       // pmin = pmin + pmin_lo exactly as float-float
    float lnp_top, inv_dln;       // ln(p) bin origin and inverse width
    float key_mx, key_my;         // float32 cell-key margins [cells]; > 0.25 disables the fast path
    const float* plev;            // [nz]    float levels
    const float* inv_dp;          // [nz]    1 / (plev[k] - plev[k+1])
    const int16_t* kguess;        // [nbins] first-guess level index per ln(p) bin
    // float64 copies for the exact cell keys of the sort
    double lon0_d, dlon_d, lat0_d, dlat_d, pmin_d, pmax_d;
    const double* plev_d;         // [nz]
};

// One met slot: records [lat][lon][level] x 4 values, scales [4][nz].
struct MetView {
    const void* rec;
    const float* scales;
};

// Both slots interleaved, the layout the particle kernels gather from: per grid
// point ([lat][lon][level]) the pairs (slot 0, slot 1) of u, v, omega, T --
// 8 float32 (32 B) or 8 16-bit codes (16 B) -- so that one load brings a
// corner's values on both snapshots, already paired.  Lane s is written when
// slot s is loaded; scales[s] are slot s's scales (16-bit storage).
struct MetPair {
    const void* rec;
    const float* scales[2];
};

// The particle arrays (null entries are absent) and their copies in the
// sort workspace: `part` is sorted in place, `copy` holds the unsorted state.
struct Arrays {
    double* d[3];      // lon, lat, p
    uint32_t* u[2];    // id, release
    float* f[3];       // up, vp, wp
};

// Hand-off from the fused step to the sort (keys == nullptr: none).  The
// launch writes every particle's final state to `copy` instead of the particle
// arrays, its cell key to keys[i] and adds it to the first-digit histogram
// hist[digit * ntiles + i / 1024] (zeroed beforehand).
struct SortEmit {
    Arrays copy;
    uint32_t* keys;
    uint32_t* hist;
    int ntiles;
};

// Arguments of the particle kernels (advect / diffuse / step).
struct StepArgs {
    Geo geo;
    MetPair mp;                   // both snapshots, interleaved (lane = slot)
    int64_t n;
    double* lon;
    double* lat;
    double* p;
    const uint32_t* id;
    const uint32_t* release;      // may be null
    float* up;
    float* vp;
    float* wp;
    const int2* win;              // per-release active step window, or null
    const uint8_t* mask;          // particles with mask[i] == 0 are left untouched, or null
    int n_rel;
    int nsteps;
    float dt, half_dt, kdeg;      // kdeg = 180 / (pi R)  [deg per metre]
    float hk, dk;                 // float products half_dt * kdeg and dt * kdeg
    int turb, meso;
    float sh, sv, inv_H;          // sqrt(2 Dx dt), sqrt(2 Dz dt), 1/H
    float r_ar, a_ar;             // AR(1) coefficient r and sqrt(1 - r^2) f
    uint32_t key0, key1;          // Philox key = seed
    uint32_t ks[20];              // Philox key schedule: round r uses (ks[2r], ks[2r+1])
    uint64_t step0;
    SortEmit emit;
    // time weights of lanes (slot 0, slot 1) at t_n and at t_n + dt/2: step q uses
    // wt[4q], wt[4q + 1] and wt[4q + 2], wt[4q + 3]
    float wt[4 * kMaxStepsPerLaunch];
};

// MODE_STEP_FULL is MODE_STEP with both diffusion parts on, resolved at compile
// time (the launcher picks it); the C ABI passes only the first three.
enum Mode { MODE_ADVECT = 0, MODE_DIFFUSE = 1, MODE_STEP = 2, MODE_STEP_FULL = 3 };

// Process-wide count of kernels this library has launched (inspection only).
void note_launches(int n);

// ---- launchers (each returns a cudaError_t of the launch) -------------------
// Blocks of `block` threads for a grid-stride launch over n items: one thread per
// item, but at most per_sm blocks per SM, so that each block fills its shared
// tables (levels, key tables) once for many items.
inline int strided_grid(int64_t n, int block, int per_sm) {
    int64_t b = (n + block - 1) / block;
    if (b < 1) b = 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0 && b > (int64_t)sms * per_sm)
        b = (int64_t)sms * per_sm;
    else
        (void)cudaGetLastError();
    return (int)(b > (1 << 20) ? (1 << 20) : b);
}

// schedule: 0 one particle per thread, 1 one wave of resident blocks, k >= 2 k particles per thread
cudaError_t launch_transport(int storage, int mode, const StepArgs& a, int grid, int variant,
                             int schedule, cudaStream_t s);
cudaError_t launch_windows(const double* ts, const double* te, int nrel, double t, double dt,
                           int n_begin, int nsteps, int2* out, cudaStream_t s);
cudaError_t launch_interp(int storage, const Geo& g, MetPair mp, float w_lane0, float w_lane1, int64_t n,
                          const double* lon, const double* lat, const double* p, float* ou,
                          float* ov, float* ow, float* ovar, cudaStream_t s);
cudaError_t launch_sample(int storage, const Geo& g, MetView m0, MetView m1, float w, int64_t n,
                          const double* lon, const double* lat, const double* p, float* out, cudaStream_t s);
cudaError_t launch_sedi(int storage, const Geo& g, MetView m0, MetView m1, int64_t n, const double* lon,
                        const double* lat, double* p, const float* radius, const float* rho_p, int nsteps,
                        float dt, float w0, float dw, cudaStream_t s);
cudaError_t launch_grid_counts(const Geo& g, int64_t n, const double* lon, const double* lat,
                               const double* p, uint32_t* counts, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out,
                          float* normals, cudaStream_t s);

// Packs one snapshot into slot records `rec` (+ scales) and into lane lane0
// of the interleaved pair records pairs0 and lane lane1 of pairs1 (the two
// slot pairs the slot belongs to).
cudaError_t launch_copy_probe(const void* src, void* dst, size_t bytes, int reps, int num_sms, cudaStream_t s);
cudaError_t launch_pack(int storage, int nvars, const float* u, const float* v, const float* w,
                        const float* T, int nx, int ny, int nz, void* rec, float* scales, void* pairs0,
                        int lane0, void* pairs1, int lane1, cudaStream_t s);

size_t sort_workspace_bytes(int64_t n);
cudaError_t launch_cell_keys(const Geo& g, int64_t n, const double* lon, const double* lat,
                             const double* p, uint32_t* keys, cudaStream_t s);
cudaError_t run_sort(const Geo& g, const mptrac_particles& P, void* ws, int key_bits,
                     cudaStream_t s);
// The hand-off arguments for the fused step over P with workspace ws (its
// first-digit histograms zeroed on s), and the radix passes that follow it.
cudaError_t sort_emit_args(const mptrac_particles& P, void* ws, SortEmit& out, cudaStream_t s);
cudaError_t sort_after_emit(const mptrac_particles& P, void* ws, int key_bits, cudaStream_t s);
// As run_sort, but particles whose release is inactive at time t (window from
// ts/te, or release index >= nrel) get the key 2^key_bits, after every cell key.
cudaError_t run_sort_at(const Geo& g, const mptrac_particles& P, void* ws, int key_bits, double t,
                        const double* ts, const double* te, int nrel, cudaStream_t s);

// ---- learned surrogate (surrogate.cu) ------------------------------------
struct Surrogate {
    int64_t max_batch = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr;
    float* b3p = nullptr;
    float *mu_x = nullptr, *isd_x = nullptr, *mu_y = nullptr, *isd_y = nullptr, *sd_y = nullptr;
    __nv_bfloat16 *Xh = nullptr, *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Yh = nullptr, *Xraw = nullptr;
    uint8_t* env = nullptr;
    float* loss_tmp = nullptr;
    int* status = nullptr;       // set by a fused-inference kernel whose bounded wait gave up
    int kernel = MPTRAC_SURR_KERNEL_TCGEN05;
};


cudaError_t surr_alloc(Surrogate& S, int64_t max_batch);
void surr_free(Surrogate& S);
cudaError_t surr_cast(Surrogate& S, cudaStream_t s);
cudaError_t surr_forward(Surrogate& S, const float* X, int64_t B, cudaStream_t s);
cudaError_t surr_backward(Surrogate& S, const float* Yt, int64_t B, float* loss, cudaStream_t s);
cudaError_t surr_adam(Surrogate& S, float lr, int step, cudaStream_t s);
cudaError_t launch_surr_features(int storage, const Geo& g, MetView m0, MetView m1, int64_t n,
                                 const double* lon, const double* lat, const double* p, float w,
                                 float* X, cudaStream_t s);
cudaError_t launch_surr_targets(int64_t n, const double* lon0, const double* lat0, const double* p0,
                                const double* lon1, const double* lat1, const double* p1, float* Y,
                                cudaStream_t s);
cudaError_t launch_colstats(const float* D, int64_t n, int ncol, double* mean, double* sd, double sd_min,
                            cudaStream_t s);
cudaError_t launch_surr_fused(int storage, Surrogate& S, const Geo& g, MetView m0, MetView m1, int64_t n,
                              double* lon, double* lat, double* p, float w, int window_ok, uint8_t* fallback,
                              uint64_t* fallback_count, double lon0, cudaStream_t s);


}  // namespace mptrac
