// C ABI of libmptrac (declared in include/mptrac.h): context management,
// host-side argument validation and kernel dispatch.  Every entry point
// validates before it launches; errors are reported as status codes plus a
// thread-local message, never as exceptions or device faults.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace mptrac;

constexpr int kSlots = MPTRAC_NUM_SLOTS;
static_assert(kSlots == 3, "the pair buffers are indexed by a + b - 1");

struct mptrac_ctx {
    int device = 0;
    int num_sms = 0;
    int nx = 0, ny = 0, nz = 0, storage = 0, nvars = 3;
    double lon0 = 0, dlon = 0, lat0 = 0, dlat = 0;
    std::vector<double> plev;
    float* d_plev = nullptr;
    float* d_invdp = nullptr;
    int16_t* d_kguess = nullptr;
    double* d_plev_d = nullptr;
    void* d_met[kSlots] = {};
    // slots a < b interleaved, lane 0 = slot a: d_pair[a + b - 1], read by the particle kernels
    void* d_pair[kSlots] = {};
    float* d_scales[kSlots] = {};
    double t_slot[kSlots] = {};
    bool loaded[kSlots] = {};
    size_t rec_bytes = 0;
    float* d_staging = nullptr;
    double* d_rel_ts = nullptr;
    double* d_rel_te = nullptr;
    int2* d_win = nullptr;
    int n_rel = 0;
    int key_bits = 0;
    int launch_variant = 0;
    int schedule = 0;   // see mptrac_set_launch
    Geo geo{};
};

namespace {

thread_local char g_err[1024] = "";
std::atomic<uint64_t> g_launches{0};

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int ok() {
    g_err[0] = '\0';
    return MPTRAC_OK;
}

#define MPTRAC_CUDA(call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (void)cudaGetLastError();                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? MPTRAC_E_OOM : MPTRAC_E_CUDA,      \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                     \
        }                                                                                    \
    } while (0)

// A pointer the device can dereference: device, managed or registered host memory.
bool device_accessible(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
           at.type == cudaMemoryTypeHost;
}

constexpr double kRadius = 6371000.0;
constexpr double kPi = 3.14159265358979323846;

void free_ctx(mptrac_ctx* c) {
    void* ptrs[] = {c->d_plev, c->d_invdp, c->d_kguess, c->d_plev_d, c->d_met[0], c->d_met[1], c->d_met[2],
                    c->d_pair[0], c->d_pair[1], c->d_pair[2], c->d_scales[0], c->d_scales[1], c->d_scales[2],
                    c->d_staging, c->d_rel_ts, c->d_rel_te, c->d_win};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

// Makes `dev` the calling thread's current device for the guard's lifetime and
// then restores the caller's: an object's memory and kernels live on the
// device it was created on, whatever device the caller has current.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        if (cur == dev) return;
        if (cudaSetDevice(dev) == cudaSuccess) prev = cur;
        else (void)cudaGetLastError();
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

int check_particles(const mptrac_particles* P, bool need_meso) {
    if (!P) return fail(MPTRAC_E_INVALID_ARG, "particles descriptor is NULL");
    if (P->n < 0 || P->n > 0x7FFFFFFF) return fail(MPTRAC_E_INVALID_ARG, "particle count %lld out of range [0, 2^31-1]", (long long)P->n);
    if (P->n == 0) return MPTRAC_OK;
    const void* req[] = {P->lon, P->lat, P->p, P->id};
    const char* names[] = {"lon", "lat", "p", "id"};
    for (int q = 0; q < 4; ++q)
        if (!device_accessible(req[q]))
            return fail(MPTRAC_E_INVALID_ARG, "particles.%s is NULL or not device memory", names[q]);
    if (P->release && !device_accessible(P->release))
        return fail(MPTRAC_E_INVALID_ARG, "particles.release is not device memory");
    const void* meso[] = {P->up, P->vp, P->wp};
    const char* mnames[] = {"up", "vp", "wp"};
    for (int q = 0; q < 3; ++q) {
        if (meso[q] && !device_accessible(meso[q]))
            return fail(MPTRAC_E_INVALID_ARG, "particles.%s is not device memory", mnames[q]);
        if (need_meso && !meso[q])
            return fail(MPTRAC_E_INVALID_ARG, "particles.%s is NULL but mesoscale diffusion is on", mnames[q]);
    }
    return MPTRAC_OK;
}

// The two loaded slots, consecutive in time, whose interval [t0, t1] contains
// [tb, te] (to 1e-9 of the interval): s0 the earlier.  E_NOT_INIT without two
// loaded slots of different times, E_TIME_RANGE when no interval contains it.
int bracket_slots(const mptrac_ctx* c, double tb, double te, int& s0, int& s1) {
    int idx[kSlots], m = 0;
    for (int q = 0; q < kSlots; ++q)
        if (c->loaded[q]) idx[m++] = q;
    for (int a = 1; a < m; ++a)   // insertion sort by time
        for (int b = a; b > 0 && c->t_slot[idx[b]] < c->t_slot[idx[b - 1]]; --b) std::swap(idx[b], idx[b - 1]);
    bool interval = false;
    for (int q = 0; q + 1 < m; ++q) {
        const double t0 = c->t_slot[idx[q]], t1 = c->t_slot[idx[q + 1]];
        if (!(t1 > t0)) continue;
        interval = true;
        const double tol = 1e-9 * (t1 - t0);
        if (tb >= t0 - tol && te <= t1 + tol) {
            s0 = idx[q];
            s1 = idx[q + 1];
            return MPTRAC_OK;
        }
    }
    if (!interval)
        return fail(MPTRAC_E_NOT_INIT, "two met slots with different times must be loaded (%d loaded)", m);
    return fail(MPTRAC_E_TIME_RANGE, "[%.9g, %.9g] lies in no interval of the loaded snapshots", tb, te);
}

// The pair buffer of slots s and o, and the lane slot s has in it.
void* pair_buffer(const mptrac_ctx* c, int s, int o) { return c->d_pair[std::min(s, o) + std::max(s, o) - 1]; }
int pair_lane(int s, int o) { return s < o ? 0 : 1; }

// The interleaved records of slots s0 and s1 (lane 0 = the lower slot index)
// and the lane weights for time fraction w from the earlier slot s0 to s1.
MetPair pair_of(const mptrac_ctx* c, int s0, int s1) {
    const int a = std::min(s0, s1), b = std::max(s0, s1);
    return MetPair{c->d_pair[a + b - 1], {c->d_scales[a], c->d_scales[b]}};
}

// Time weights of the pair lanes for the time fraction w from the earlier
// slot s0 to the later slot s1 (lane 0 holds the lower slot index).
void lane_weights(int s0, int s1, double w, float& lane0, float& lane1) {
    const float early = (float)(1.0 - w), late = (float)w;
    lane0 = s0 < s1 ? early : late;
    lane1 = s0 < s1 ? late : early;
}

int run_transport(mptrac_ctx* c, const mptrac_particles* P, double t, double dt,
                  const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps,
                  uintptr_t stream, int mode, const uint8_t* mask = nullptr, const SortEmit* emit = nullptr) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MPTRAC_E_INVALID_ARG, "dt must be finite and > 0 (got %g)", dt);
    if (!std::isfinite(t)) return fail(MPTRAC_E_INVALID_ARG, "t must be finite");
    if (nsteps < 0) return fail(MPTRAC_E_INVALID_ARG, "nsteps must be >= 0 (got %d)", nsteps);
    bool turb = false, meso = false;
    if (mode != MODE_ADVECT) {
        if (!prm) return fail(MPTRAC_E_INVALID_ARG, "diffusion parameters are NULL");
        turb = prm->turb != 0;
        meso = prm->meso != 0;
        if (!(prm->dx >= 0) || !(prm->dz >= 0) || !(prm->meso_f >= 0) || !(prm->scale_height > 0) ||
            !std::isfinite(prm->dx) || !std::isfinite(prm->dz) || !std::isfinite(prm->meso_f) ||
            !std::isfinite(prm->scale_height))
            return fail(MPTRAC_E_INVALID_ARG, "diffusion parameters out of range");
    }
    int rc = check_particles(P, meso);
    if (rc) return rc;
    int s0, s1;
    const double tend = t + (double)nsteps * dt;
    if ((rc = bracket_slots(c, t, tend, s0, s1))) return rc;
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    if (P->n == 0 || nsteps == 0) return ok();
    // the fused step with both diffusion terms off is exactly the advection kernel
    if (mode == MODE_STEP && !turb && !meso) mode = MODE_ADVECT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.geo = c->geo;
    a.mp = pair_of(c, s0, s1);
    a.n = P->n;
    a.lon = P->lon;
    a.lat = P->lat;
    a.p = P->p;
    a.id = P->id;
    a.release = P->release;
    a.up = P->up;
    a.vp = P->vp;
    a.wp = P->wp;
    const bool use_win = P->release && c->n_rel > 0;
    a.win = use_win ? c->d_win : nullptr;
    a.mask = mask;
    a.n_rel = c->n_rel;
    a.dt = (float)dt;
    a.half_dt = (float)(0.5 * dt);
    a.kdeg = (float)(180.0 / (kPi * kRadius));
    {
        // float products, rounded once like the device multiplication they replace
        volatile float hd = a.half_dt, dd = a.dt, kd = a.kdeg;
        a.hk = hd * kd;
        a.dk = dd * kd;
    }
    a.turb = turb;
    a.meso = meso;
    if (mode != MODE_ADVECT) {
        a.sh = (float)std::sqrt(2.0 * prm->dx * dt);
        a.sv = (float)std::sqrt(2.0 * prm->dz * dt);
        a.inv_H = (float)(1.0 / prm->scale_height);
        double r = 1.0 - 2.0 * dt / (t1 - t0);
        r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
        a.r_ar = (float)r;
        a.a_ar = (float)(std::sqrt(1.0 - r * r) * prm->meso_f);
    }
    a.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {   // Philox4x32 key bumps (Salmon et al., SC'11)
        a.ks[2 * r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
        a.ks[2 * r + 1] = a.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    const int grid = (int)std::min<int64_t>((P->n + kBlock - 1) / kBlock, (int64_t)1 << 20);
    for (int n0 = 0; n0 < nsteps; n0 += kMaxStepsPerLaunch) {
        const int cnt = std::min(kMaxStepsPerLaunch, nsteps - n0);
        a.nsteps = cnt;
        a.step0 = step0 + (uint64_t)n0;
        for (int q = 0; q < cnt; ++q) {
            const double tn = t + (double)(n0 + q) * dt;
            lane_weights(s0, s1, (tn - t0) / (t1 - t0), a.wt[4 * q], a.wt[4 * q + 1]);
            lane_weights(s0, s1, (tn + 0.5 * dt - t0) / (t1 - t0), a.wt[4 * q + 2], a.wt[4 * q + 3]);
        }
        if (use_win) MPTRAC_CUDA(launch_windows(c->d_rel_ts, c->d_rel_te, c->n_rel, t, dt, n0, cnt, c->d_win, st));
        // the last launch hands its results to the sort, if one follows
        a.emit = (emit && n0 + cnt >= nsteps) ? *emit : SortEmit{};
        MPTRAC_CUDA(launch_transport(c->storage, mode, a, grid, c->launch_variant, c->schedule, st));
    }
    return ok();
}

}  // namespace

namespace mptrac {
void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace mptrac

extern "C" {

uint64_t mptrac_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int mptrac_copy_probe(const void* src, void* dst, size_t bytes, int reps, uintptr_t stream) {
    if (reps < 1) return fail(MPTRAC_E_INVALID_ARG, "reps must be >= 1");
    if (bytes % 16 || (reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(dst) & 15))
        return fail(MPTRAC_E_INVALID_ARG, "bytes must be a multiple of 16 and both pointers 16-byte aligned");
    if (bytes == 0) return ok();
    if (!device_accessible(src) || !device_accessible(dst))
        return fail(MPTRAC_E_INVALID_ARG, "src and dst must be device memory");
    int dev = 0, sms = 0;
    MPTRAC_CUDA(cudaGetDevice(&dev));
    MPTRAC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MPTRAC_CUDA(launch_copy_probe(src, dst, bytes, reps, sms, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_init_grid(mptrac_ctx** out, const mptrac_grid_desc* g) {
    if (!out || !g) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || g->nz > MPTRAC_MAX_NZ)
        return fail(MPTRAC_E_INVALID_ARG, "grid size %d x %d x %d out of range", g->nx, g->ny, g->nz);
    const int64_t npts = (int64_t)g->nx * g->ny * g->nz;
    if (npts >= ((int64_t)1 << 31)) return fail(MPTRAC_E_INVALID_ARG, "grid has %lld points (limit 2^31-1)", (long long)npts);
    if (!(g->dlon > 0) || !(g->dlat > 0) || !std::isfinite(g->lon0) || !std::isfinite(g->lat0))
        return fail(MPTRAC_E_INVALID_ARG, "bad grid spacing or origin");
    if (std::fabs(g->nx * g->dlon - 360.0) > 1e-9 * 360.0)
        return fail(MPTRAC_E_INVALID_ARG, "nx * dlon = %.12g, must be 360 (periodic longitude)", g->nx * g->dlon);
    if ((double)(float)g->lon0 != g->lon0 || (double)(float)g->lat0 != g->lat0)
        return fail(MPTRAC_E_INVALID_ARG, "lon0 and lat0 must be exactly representable in float32");
    if (g->storage < MPTRAC_FP32 || g->storage > MPTRAC_FP16) return fail(MPTRAC_E_INVALID_ARG, "unknown storage %d", g->storage);
    if (g->nvars != 3 && g->nvars != 4) return fail(MPTRAC_E_INVALID_ARG, "nvars must be 3 or 4");
    if (!g->plev) return fail(MPTRAC_E_INVALID_ARG, "plev is NULL");
    for (int k = 0; k < g->nz; ++k) {
        if (!(g->plev[k] > 0) || !std::isfinite(g->plev[k])) return fail(MPTRAC_E_INVALID_ARG, "plev[%d] must be finite and > 0", k);
        if (k && !(g->plev[k] < g->plev[k - 1])) return fail(MPTRAC_E_INVALID_ARG, "plev must be strictly decreasing (level %d)", k);
    }
    mptrac_ctx* c = new (std::nothrow) mptrac_ctx();
    if (!c) return fail(MPTRAC_E_OOM, "host allocation failed");
    c->nx = g->nx; c->ny = g->ny; c->nz = g->nz;
    c->lon0 = g->lon0; c->dlon = g->dlon; c->lat0 = g->lat0; c->dlat = g->dlat;
    c->storage = g->storage; c->nvars = g->nvars;
    c->plev.assign(g->plev, g->plev + g->nz);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return fail(MPTRAC_E_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    const int nz = g->nz;
    std::vector<float> plev_f(nz), invdp(nz, 0.f);
    for (int k = 0; k < nz; ++k) plev_f[k] = (float)g->plev[k];
    for (int k = 0; k + 1 < nz; ++k) invdp[k] = (float)(1.0 / ((double)plev_f[k] - (double)plev_f[k + 1]));
    const double ln_top = std::log(g->plev[nz - 1]), ln_bot = std::log(g->plev[0]);
    const int nbins = kGuessBins;
    const double inv_dln = nbins / (ln_bot - ln_top);
    std::vector<int16_t> kg(nbins);
    for (int b = 0; b < nbins; ++b) {
        const double pc = std::exp(ln_top + (b + 0.5) / inv_dln);
        int cnt = 0;
        for (int k = 0; k < nz; ++k) cnt += (plev_f[k] >= pc);
        int k = cnt - 1;
        k = k < 0 ? 0 : (k > nz - 2 ? nz - 2 : k);
        kg[b] = (int16_t)k;
    }
    c->rec_bytes = (size_t)npts * (g->storage == MPTRAC_FP32 ? 16 : 8);
    // npts < 2^31 (checked above), so key_bits <= 31: cell keys and the release-aware sort's
    // inactive key 2^key_bits fit a 32-bit word.
    c->key_bits = 0;
    while (c->key_bits < 31 && ((uint64_t)1 << c->key_bits) < (uint64_t)npts) ++c->key_bits;

    auto alloc = [&](void** p, size_t bytes) -> int {
        cudaError_t ee = cudaMalloc(p, bytes);
        if (ee != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ee == cudaErrorMemoryAllocation ? MPTRAC_E_OOM : MPTRAC_E_CUDA,
                        "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(ee));
        }
        return MPTRAC_OK;
    };
    int rc = MPTRAC_OK;
    if (!rc) rc = alloc((void**)&c->d_plev, nz * sizeof(float));
    if (!rc) rc = alloc((void**)&c->d_invdp, nz * sizeof(float));
    if (!rc) rc = alloc((void**)&c->d_kguess, nbins * sizeof(int16_t));
    if (!rc) rc = alloc((void**)&c->d_plev_d, nz * sizeof(double));
    for (int s = 0; s < kSlots && !rc; ++s) {
        rc = alloc(&c->d_met[s], c->rec_bytes);
        if (!rc) rc = alloc((void**)&c->d_scales[s], 4 * nz * sizeof(float));
        if (!rc) rc = alloc(&c->d_pair[s], 2 * c->rec_bytes);
        if (!rc && cudaMemset(c->d_pair[s], 0, 2 * c->rec_bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = fail(MPTRAC_E_CUDA, "clearing the pair records failed");
        }
    }
    if (rc) {
        free_ctx(c);
        return rc;
    }
    e = cudaMemcpy(c->d_plev, plev_f.data(), nz * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_invdp, invdp.data(), nz * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_kguess, kg.data(), nbins * sizeof(int16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_plev_d, g->plev, nz * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_ctx(c);
        return fail(MPTRAC_E_CUDA, "table upload failed: %s", cudaGetErrorString(e));
    }
    Geo& G = c->geo;
    G.nx = g->nx; G.ny = g->ny; G.nz = nz; G.nbins = nbins;
    G.lon0 = (float)g->lon0;
    G.inv_dlon = (float)(1.0 / g->dlon);
    G.inv_dlon_lo = (float)(1.0 / g->dlon - (double)G.inv_dlon);
    G.lat0 = (float)g->lat0;
    G.inv_dlat = (float)(1.0 / g->dlat);
    G.inv_dlat_lo = (float)(1.0 / g->dlat - (double)G.inv_dlat);
    G.dn = (float)(90.0 - g->lat0);
    G.dn_lo = (float)((90.0 - g->lat0) - (double)G.dn);
    G.ds = (float)(-90.0 - g->lat0);
    G.ds_lo = (float)((-90.0 - g->lat0) - (double)G.ds);
    G.dmid = -G.lat0;
    const double pmin = g->plev[nz - 1], pmax = g->plev[0];
    G.pmin = (float)pmin;
    G.pmin_lo = (float)(pmin - (double)G.pmin);
    G.pmax = (float)pmax;
    G.pmax_lo = (float)(pmax - (double)G.pmax);
    G.lnp_top = (float)ln_top;
    // bound of the float32 cell-coordinate error: truncation of lon/lat to
    // float (2^-23 |lon|), rounding of the subtraction (2^-24 |lon - lon0|), of
    // 1/dlon and of the product (2^-24 |x| each), times 2 for safety
    G.key_mx = (float)(2.0 * (std::ldexp(2.0 * std::fabs(g->lon0) + 1080.0, -24) / g->dlon + std::ldexp((double)g->nx, -23)));
    G.key_my = (float)(2.0 * (std::ldexp(2.0 * std::fabs(g->lat0) + 540.0, -24) / g->dlat + std::ldexp((double)g->ny, -23)));
    G.inv_dln = (float)inv_dln;
    G.plev = c->d_plev;
    G.inv_dp = c->d_invdp;
    G.kguess = c->d_kguess;
    G.lon0_d = g->lon0; G.dlon_d = g->dlon; G.lat0_d = g->lat0; G.dlat_d = g->dlat;
    G.pmin_d = pmin; G.pmax_d = pmax;
    G.plev_d = c->d_plev_d;
    *out = c;
    return ok();
}

int mptrac_destroy(mptrac_ctx* ctx) {
    if (!ctx) return ok();
    DeviceGuard device_guard(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    free_ctx(ctx);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(MPTRAC_E_CUDA, "device error while destroying context: %s", cudaGetErrorString(e));
    }
    return ok();
}

const char* mptrac_last_error(const mptrac_ctx*) { return g_err; }

int mptrac_load_met(mptrac_ctx* c, int slot, double t, const float* u, const float* v,
                    const float* omega, const float* T, int src_is_device, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (slot < 0 || slot >= kSlots) return fail(MPTRAC_E_INVALID_ARG, "slot must be 0, 1 or 2 (got %d)", slot);
    if (!std::isfinite(t)) return fail(MPTRAC_E_INVALID_ARG, "t must be finite");
    if (!u || !v || !omega) return fail(MPTRAC_E_INVALID_ARG, "u, v and omega must not be NULL");
    if (c->nvars == 4 && !T) return fail(MPTRAC_E_INVALID_ARG, "T must not be NULL when nvars == 4");
    if (c->nvars == 3) T = nullptr;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t npts = (size_t)c->nx * c->ny * c->nz;
    const float* src[4] = {u, v, omega, T};
    if (src_is_device) {
        for (int q = 0; q < c->nvars; ++q)
            if (!device_accessible(src[q])) return fail(MPTRAC_E_INVALID_ARG, "met variable %d is not device memory", q);
    } else {
        if (!c->d_staging) {
            cudaError_t e = cudaMalloc((void**)&c->d_staging, 4 * npts * sizeof(float));
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                c->d_staging = nullptr;
                return fail(MPTRAC_E_OOM, "staging allocation failed: %s", cudaGetErrorString(e));
            }
        }
        for (int q = 0; q < c->nvars; ++q) {
            float* dst = c->d_staging + q * npts;
            MPTRAC_CUDA(cudaMemcpyAsync(dst, src[q], npts * sizeof(float), cudaMemcpyHostToDevice, st));
            src[q] = dst;
        }
    }
    MPTRAC_CUDA(launch_pack(c->storage, c->nvars, src[0], src[1], src[2], src[3], c->nx, c->ny, c->nz,
                            c->d_met[slot], c->d_scales[slot], pair_buffer(c, slot, (slot + 1) % kSlots),
                            pair_lane(slot, (slot + 1) % kSlots), pair_buffer(c, slot, (slot + 2) % kSlots),
                            pair_lane(slot, (slot + 2) % kSlots), st));
    c->t_slot[slot] = t;
    c->loaded[slot] = true;
    return ok();
}

int mptrac_set_releases(mptrac_ctx* c, int n, const double* ts, const double* te) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (n < 0 || n > MPTRAC_MAX_RELEASES) return fail(MPTRAC_E_INVALID_ARG, "release count %d out of range", n);
    if (n > 0 && (!ts || !te)) return fail(MPTRAC_E_INVALID_ARG, "release times are NULL");
    for (int r = 0; r < n; ++r)
        if (std::isnan(ts[r]) || std::isnan(te[r])) return fail(MPTRAC_E_INVALID_ARG, "release %d has NaN times", r);
    void* old[] = {c->d_rel_ts, c->d_rel_te, c->d_win};
    for (void* p : old)
        if (p) MPTRAC_CUDA(cudaFree(p));
    c->d_rel_ts = c->d_rel_te = nullptr;
    c->d_win = nullptr;
    c->n_rel = 0;
    if (n == 0) return ok();
    MPTRAC_CUDA(cudaMalloc((void**)&c->d_rel_ts, n * sizeof(double)));
    MPTRAC_CUDA(cudaMalloc((void**)&c->d_rel_te, n * sizeof(double)));
    MPTRAC_CUDA(cudaMalloc((void**)&c->d_win, n * sizeof(int2)));
    MPTRAC_CUDA(cudaMemcpy(c->d_rel_ts, ts, n * sizeof(double), cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemcpy(c->d_rel_te, te, n * sizeof(double), cudaMemcpyHostToDevice));
    c->n_rel = n;
    return ok();
}

int mptrac_advect(mptrac_ctx* c, const mptrac_particles* P, double t, double dt, int nsteps,
                  uintptr_t stream) {
    return run_transport(c, P, t, dt, nullptr, 0, 0, nsteps, stream, MODE_ADVECT);
}

int mptrac_diffuse(mptrac_ctx* c, const mptrac_particles* P, double t, double dt,
                   const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps,
                   uintptr_t stream) {
    return run_transport(c, P, t, dt, prm, seed, step0, nsteps, stream, MODE_DIFFUSE);
}

int mptrac_step(mptrac_ctx* c, const mptrac_particles* P, double t, double dt,
                const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps,
                uintptr_t stream) {
    return run_transport(c, P, t, dt, prm, seed, step0, nsteps, stream, MODE_STEP);
}

int check_workspace(const mptrac_particles* P, const void* ws, size_t ws_bytes) {
    const size_t need = sort_workspace_bytes(P->n);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need)
        return fail(MPTRAC_E_WORKSPACE, "sort workspace must be 256-byte aligned device memory of >= %zu bytes (got %p, %zu)", need, ws, ws_bytes);
    if (!device_accessible(ws)) return fail(MPTRAC_E_WORKSPACE, "sort workspace is not device memory");
    return MPTRAC_OK;
}

int mptrac_step_handoff(mptrac_ctx* c, const mptrac_particles* P, double t, double dt,
                        const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps, void* ws,
                        size_t ws_bytes, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (nsteps < 1) return fail(MPTRAC_E_INVALID_ARG, "nsteps must be >= 1 for a hand-off (got %d)", nsteps);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n == 0) return run_transport(c, P, t, dt, prm, seed, step0, nsteps, stream, MODE_STEP);
    if ((rc = check_workspace(P, ws, ws_bytes))) return rc;
    SortEmit e{};
    MPTRAC_CUDA(sort_emit_args(*P, ws, e, reinterpret_cast<cudaStream_t>(stream)));
    return run_transport(c, P, t, dt, prm, seed, step0, nsteps, stream, MODE_STEP, nullptr, &e);
}

int mptrac_sort_handoff(mptrac_ctx* c, const mptrac_particles* P, void* ws, size_t ws_bytes,
                        uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n == 0) return ok();
    if ((rc = check_workspace(P, ws, ws_bytes))) return rc;
    MPTRAC_CUDA(sort_after_emit(*P, ws, c->key_bits, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_step_sort(mptrac_ctx* c, const mptrac_particles* P, double t, double dt,
                     const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps, void* ws,
                     size_t ws_bytes, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    if (nsteps == 0) {   // nothing to hand off: the arguments are checked, then a plain sort
        int rc = run_transport(c, P, t, dt, prm, seed, step0, nsteps, stream, MODE_STEP);
        return rc ? rc : mptrac_sort(c, P, ws, ws_bytes, stream);
    }
    int rc = mptrac_step_handoff(c, P, t, dt, prm, seed, step0, nsteps, ws, ws_bytes, stream);
    return rc ? rc : mptrac_sort_handoff(c, P, ws, ws_bytes, stream);
}

size_t mptrac_sort_workspace_bytes(const mptrac_ctx*, int64_t n) {
    return sort_workspace_bytes(n < 0 ? 0 : n);
}

int mptrac_sort(mptrac_ctx* c, const mptrac_particles* P, void* ws, size_t ws_bytes,
                uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n == 0) return ok();
    const size_t need = sort_workspace_bytes(P->n);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need)
        return fail(MPTRAC_E_WORKSPACE, "sort workspace must be 256-byte aligned device memory of >= %zu bytes (got %p, %zu)", need, ws, ws_bytes);
    if (!device_accessible(ws)) return fail(MPTRAC_E_WORKSPACE, "sort workspace is not device memory");
    MPTRAC_CUDA(run_sort(c->geo, *P, ws, c->key_bits, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_sort_at(mptrac_ctx* c, const mptrac_particles* P, double t, void* ws, size_t ws_bytes,
                   uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (!std::isfinite(t)) return fail(MPTRAC_E_INVALID_ARG, "t must be finite");
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n == 0) return ok();
    const size_t need = sort_workspace_bytes(P->n);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need)
        return fail(MPTRAC_E_WORKSPACE, "sort workspace must be 256-byte aligned device memory of >= %zu bytes (got %p, %zu)", need, ws, ws_bytes);
    if (!device_accessible(ws)) return fail(MPTRAC_E_WORKSPACE, "sort workspace is not device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!P->release || c->n_rel == 0) {
        MPTRAC_CUDA(run_sort(c->geo, *P, ws, c->key_bits, st));
    } else {
        MPTRAC_CUDA(run_sort_at(c->geo, *P, ws, c->key_bits, t, c->d_rel_ts, c->d_rel_te, c->n_rel, st));
    }
    return ok();
}

int mptrac_set_launch(mptrac_ctx* c, int variant, int schedule) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (variant < 0 || variant > 6) return fail(MPTRAC_E_INVALID_ARG, "launch variant must be 0..6 (got %d)", variant);
    if (schedule < 0 || schedule > 64)
        return fail(MPTRAC_E_INVALID_ARG, "launch schedule must be 0..64 (got %d)", schedule);
    c->launch_variant = variant;
    c->schedule = schedule;
    return ok();
}

int mptrac_cell_keys(mptrac_ctx* c, const mptrac_particles* P, uint32_t* keys, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n == 0) return ok();
    if (!device_accessible(keys)) return fail(MPTRAC_E_INVALID_ARG, "keys is not device memory");
    MPTRAC_CUDA(launch_cell_keys(c->geo, P->n, P->lon, P->lat, P->p, keys, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_interp(mptrac_ctx* c, int64_t n, const double* lon, const double* lat, const double* p,
                  double t, float* ou, float* ov, float* ow, float* ovar, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (n < 0 || n > 0x7FFFFFFF) return fail(MPTRAC_E_INVALID_ARG, "n out of range");
    int s0, s1, rc;
    if ((rc = bracket_slots(c, t, t, s0, s1))) return rc;
    if (n == 0) return ok();
    const void* ptrs[] = {lon, lat, p, ou, ov, ow};
    for (const void* q : ptrs)
        if (!device_accessible(q)) return fail(MPTRAC_E_INVALID_ARG, "interp arrays must be device memory");
    if (ovar && !device_accessible(ovar)) return fail(MPTRAC_E_INVALID_ARG, "out_var is not device memory");
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    float wl0, wl1;
    lane_weights(s0, s1, (t - t0) / (t1 - t0), wl0, wl1);
    MPTRAC_CUDA(launch_interp(c->storage, c->geo, pair_of(c, s0, s1), wl0, wl1, n, lon, lat, p, ou, ov, ow, ovar,
                              reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out, float* normals,
                  uintptr_t stream) {
    if (n < 0 || n > 0x7FFFFFFF) return fail(MPTRAC_E_INVALID_ARG, "n out of range");
    if (n == 0) return ok();
    if (!device_accessible(ctr) || !device_accessible(out))
        return fail(MPTRAC_E_INVALID_ARG, "ctr and out must be device memory");
    if (normals && !device_accessible(normals)) return fail(MPTRAC_E_INVALID_ARG, "normals is not device memory");
    MPTRAC_CUDA(launch_philox(ctr, n, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), out,
                              normals, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_met_slot_info(const mptrac_ctx* c, int slot, const void** records, const float** scales,
                         double* t, size_t* bytes) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (slot < 0 || slot >= kSlots) return fail(MPTRAC_E_INVALID_ARG, "slot must be 0, 1 or 2");
    if (records) *records = c->d_met[slot];
    if (scales) *scales = c->d_scales[slot];
    if (t) *t = c->t_slot[slot];
    if (bytes) *bytes = c->rec_bytes;
    return ok();
}

int mptrac_met_slot_copy(const mptrac_ctx* c, int slot, void* rec_out, float* sc_out,
                         uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (slot < 0 || slot >= kSlots) return fail(MPTRAC_E_INVALID_ARG, "slot must be 0, 1 or 2");
    if (rec_out && !device_accessible(rec_out)) return fail(MPTRAC_E_INVALID_ARG, "records_out is not device memory");
    if (sc_out && !device_accessible(sc_out)) return fail(MPTRAC_E_INVALID_ARG, "scales_out is not device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (rec_out) MPTRAC_CUDA(cudaMemcpyAsync(rec_out, c->d_met[slot], c->rec_bytes, cudaMemcpyDeviceToDevice, st));
    if (sc_out) MPTRAC_CUDA(cudaMemcpyAsync(sc_out, c->d_scales[slot], 4 * c->nz * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return ok();
}

int mptrac_sample_met(mptrac_ctx* c, const mptrac_particles* P, double t, float* out, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    int s0, s1;
    if ((rc = bracket_slots(c, t, t, s0, s1))) return rc;
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    if (P->n == 0) return ok();
    if (!device_accessible(out)) return fail(MPTRAC_E_INVALID_ARG, "out must be device memory");
    MPTRAC_CUDA(launch_sample(c->storage, c->geo, MetView{c->d_met[s0], c->d_scales[s0]},
                              MetView{c->d_met[s1], c->d_scales[s1]}, (float)((t - t0) / (t1 - t0)), P->n,
                              P->lon, P->lat, P->p, out, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_sediment(mptrac_ctx* c, const mptrac_particles* P, const float* radius, const float* density, double t,
                    double dt, int nsteps, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (c->nvars != 4) return fail(MPTRAC_E_INVALID_ARG, "sedimentation needs temperature (nvars == 4)");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(MPTRAC_E_INVALID_ARG, "bad dt or nsteps");
    int rc = check_particles(P, false);
    if (rc) return rc;
    int s0, s1;
    if ((rc = bracket_slots(c, t, t + nsteps * dt, s0, s1))) return rc;
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    if (P->n == 0 || nsteps == 0) return ok();
    if (!device_accessible(radius) || !device_accessible(density))
        return fail(MPTRAC_E_INVALID_ARG, "radius and density must be device memory");
    MPTRAC_CUDA(launch_sedi(c->storage, c->geo, MetView{c->d_met[s0], c->d_scales[s0]},
                            MetView{c->d_met[s1], c->d_scales[s1]}, P->n, P->lon, P->lat, P->p, radius, density,
                            nsteps, (float)dt, (float)((t - t0) / (t1 - t0)), (float)(dt / (t1 - t0)),
                            reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_grid_counts(mptrac_ctx* c, const mptrac_particles* P, uint32_t* counts, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (!device_accessible(counts)) return fail(MPTRAC_E_INVALID_ARG, "counts must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    MPTRAC_CUDA(cudaMemsetAsync(counts, 0, (size_t)c->nx * c->ny * c->nz * sizeof(uint32_t), st));
    if (P->n == 0) return ok();
    MPTRAC_CUDA(launch_grid_counts(c->geo, P->n, P->lon, P->lat, P->p, counts, st));
    return ok();
}

int mptrac_advect_masked(mptrac_ctx* c, const mptrac_particles* P, const uint8_t* mask, double t,
                         double dt, int nsteps, uintptr_t stream) {
    if (P && P->n > 0 && !device_accessible(mask))
        return fail(MPTRAC_E_INVALID_ARG, "mask must be device memory");
    return run_transport(c, P, t, dt, nullptr, 0, 0, nsteps, stream, MODE_ADVECT, mask);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned surrogate: C ABI over surrogate.cu
// ---------------------------------------------------------------------------
struct mptrac_surr {
    mptrac::Surrogate S;
    int device = 0;   // the device its buffers live on
};

extern "C" {

int mptrac_surr_create(mptrac_surr** out, int64_t max_batch) {
    if (!out) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (max_batch < 64 || max_batch > (1 << 22))
        return fail(MPTRAC_E_INVALID_ARG, "max_batch must be in [64, 4194304] (got %lld)", (long long)max_batch);
    mptrac_surr* s = new (std::nothrow) mptrac_surr();
    if (!s) return fail(MPTRAC_E_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = surr_alloc(s->S, max_batch);
    if (e == cudaSuccess) {
        // identity normalisation
        std::vector<float> one(MPTRAC_SURR_KPAD, 1.f);
        e = cudaMemcpy(s->S.isd_x, one.data(), MPTRAC_SURR_KPAD * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->S.isd_y, one.data(), 8 * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->S.sd_y, one.data(), 8 * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        surr_free(s->S);
        delete s;
        return fail(e == cudaErrorMemoryAllocation ? MPTRAC_E_OOM : MPTRAC_E_CUDA, "surrogate allocation failed: %s",
                    cudaGetErrorString(e));
    }
    *out = s;
    return ok();
}

int mptrac_surr_destroy(mptrac_surr* s) {
    if (!s) return ok();
    DeviceGuard device_guard(s->device);
    cudaDeviceSynchronize();
    surr_free(s->S);
    delete s;
    return ok();
}

int mptrac_surr_set_params(mptrac_surr* s, const float* params) {
    if (!s || !params) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    DeviceGuard device_guard_s(s->device);
    MPTRAC_CUDA(cudaMemcpy(s->S.theta, params, MPTRAC_SURR_NPARAM * 4, cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemset(s->S.m, 0, MPTRAC_SURR_NPARAM * 4));
    MPTRAC_CUDA(cudaMemset(s->S.v, 0, MPTRAC_SURR_NPARAM * 4));
    MPTRAC_CUDA(surr_cast(s->S, 0));
    MPTRAC_CUDA(cudaDeviceSynchronize());
    return ok();
}

int mptrac_surr_get_params(const mptrac_surr* s, float* params) {
    if (!s || !params) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    DeviceGuard device_guard_s(s->device);
    MPTRAC_CUDA(cudaDeviceSynchronize());
    MPTRAC_CUDA(cudaMemcpy(params, s->S.theta, MPTRAC_SURR_NPARAM * 4, cudaMemcpyDeviceToHost));
    return ok();
}

int mptrac_surr_get_grads(const mptrac_surr* s, float* grads) {
    if (!s || !grads) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    DeviceGuard device_guard_s(s->device);
    MPTRAC_CUDA(cudaDeviceSynchronize());
    MPTRAC_CUDA(cudaMemcpy(grads, s->S.grad, MPTRAC_SURR_NPARAM * 4, cudaMemcpyDeviceToHost));
    return ok();
}

int mptrac_surr_set_norm(mptrac_surr* s, const float* mu_x, const float* sd_x, const float* mu_y,
                         const float* sd_y) {
    if (!s || !mu_x || !sd_x || !mu_y || !sd_y) return fail(MPTRAC_E_INVALID_ARG, "NULL argument");
    DeviceGuard device_guard_s(s->device);
    float mx[MPTRAC_SURR_KPAD], ix[MPTRAC_SURR_KPAD], my[8] = {0}, iy[8], sy[8];
    for (int c = 0; c < MPTRAC_SURR_KPAD; ++c) {
        const bool used = c < MPTRAC_SURR_NFEAT;
        if (used && !(sd_x[c] > 0.f)) return fail(MPTRAC_E_INVALID_ARG, "sd_x[%d] must be > 0", c);
        mx[c] = used ? mu_x[c] : 0.f;
        ix[c] = used ? 1.f / sd_x[c] : 1.f;
    }
    for (int c = 0; c < 8; ++c) {
        const bool used = c < MPTRAC_SURR_NOUT;
        if (used && !(sd_y[c] > 0.f)) return fail(MPTRAC_E_INVALID_ARG, "sd_y[%d] must be > 0", c);
        my[c] = used ? mu_y[c] : 0.f;
        sy[c] = used ? sd_y[c] : 1.f;
        iy[c] = 1.f / sy[c];
    }
    MPTRAC_CUDA(cudaMemcpy(s->S.mu_x, mx, sizeof(mx), cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemcpy(s->S.isd_x, ix, sizeof(ix), cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemcpy(s->S.mu_y, my, sizeof(my), cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemcpy(s->S.isd_y, iy, sizeof(iy), cudaMemcpyHostToDevice));
    MPTRAC_CUDA(cudaMemcpy(s->S.sd_y, sy, sizeof(sy), cudaMemcpyHostToDevice));
    return ok();
}

int mptrac_surr_features(mptrac_ctx* c, const mptrac_particles* P, double t, float* feat, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (c->nx < 3 || c->ny < 3 || c->nz < 3) return fail(MPTRAC_E_INVALID_ARG, "surrogate features need nx, ny, nz >= 3");
    int s0, s1;
    if ((rc = bracket_slots(c, t, t, s0, s1))) return rc;
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    if (P->n == 0) return ok();
    if (!device_accessible(feat)) return fail(MPTRAC_E_INVALID_ARG, "feat must be device memory");
    MPTRAC_CUDA(launch_surr_features(c->storage, c->geo, MetView{c->d_met[s0], c->d_scales[s0]},
                                     MetView{c->d_met[s1], c->d_scales[s1]}, P->n, P->lon, P->lat, P->p,
                                     (float)((t - t0) / (t1 - t0)), feat, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_surr_targets(int64_t n, const double* lon0, const double* lat0, const double* p0, const double* lon1,
                        const double* lat1, const double* p1, float* y, uintptr_t stream) {
    if (n < 0) return fail(MPTRAC_E_INVALID_ARG, "n < 0");
    if (n == 0) return ok();
    const void* ptrs[] = {lon0, lat0, p0, lon1, lat1, p1, y};
    for (const void* q : ptrs)
        if (!device_accessible(q)) return fail(MPTRAC_E_INVALID_ARG, "target arrays must be device memory");
    MPTRAC_CUDA(launch_surr_targets(n, lon0, lat0, p0, lon1, lat1, p1, y, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_surr_colstats(const float* data, int64_t n, int ncol, double* mean, double* sd, double sd_min,
                         uintptr_t stream) {
    if (n < 1 || ncol <= 0 || ncol > 4096) return fail(MPTRAC_E_INVALID_ARG, "bad size (n >= 1, 1 <= ncol <= 4096)");
    if (!device_accessible(data) || !device_accessible(mean) || !device_accessible(sd))
        return fail(MPTRAC_E_INVALID_ARG, "colstats arrays must be device memory");
    MPTRAC_CUDA(launch_colstats(data, n, ncol, mean, sd, sd_min, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_surr_forward(mptrac_surr* s, const float* x, int64_t n, float* y_hat, uintptr_t stream) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    if (n < 0 || n > s->S.max_batch) return fail(MPTRAC_E_INVALID_ARG, "n must be in [0, max_batch]");
    if (n == 0) return ok();
    if (!device_accessible(x) || (y_hat && !device_accessible(y_hat)))
        return fail(MPTRAC_E_INVALID_ARG, "x and y_hat must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    MPTRAC_CUDA(surr_forward(s->S, x, n, st));
    if (y_hat) MPTRAC_CUDA(cudaMemcpyAsync(y_hat, s->S.Yh, (size_t)n * 8 * 4, cudaMemcpyDeviceToDevice, st));
    return ok();
}

int mptrac_surr_grads(mptrac_surr* s, const float* x, const float* y, int64_t n, float* loss, uintptr_t stream) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    if (n <= 0 || n > s->S.max_batch) return fail(MPTRAC_E_INVALID_ARG, "n must be in [1, max_batch]");
    if (!device_accessible(x) || !device_accessible(y) || !device_accessible(loss))
        return fail(MPTRAC_E_INVALID_ARG, "x, y and loss must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    MPTRAC_CUDA(surr_forward(s->S, x, n, st));
    MPTRAC_CUDA(surr_backward(s->S, y, n, loss, st));
    return ok();
}

int mptrac_surr_train_step(mptrac_surr* s, const float* x, const float* y, int64_t n, float lr, int step,
                           float* loss, uintptr_t stream) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    if (step < 1 || !(lr > 0.f)) return fail(MPTRAC_E_INVALID_ARG, "step must be >= 1 and lr > 0");
    int rc = mptrac_surr_grads(s, x, y, n, loss, stream);
    if (rc) return rc;
    MPTRAC_CUDA(surr_adam(s->S, lr, step, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

int mptrac_surr_train_epoch(mptrac_surr* s, const float* x, const float* y, int64_t n, int64_t batch,
                            double lr_max, double lr_min, int step0, int total_steps, float* loss,
                            uintptr_t stream) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    if (batch <= 0 || batch > s->S.max_batch) return fail(MPTRAC_E_INVALID_ARG, "batch must be in [1, max_batch]");
    if (n < batch) return fail(MPTRAC_E_INVALID_ARG, "n (%lld) holds no whole batch", (long long)n);
    if (!(lr_min > 0.0) || !(lr_max >= lr_min) || !((float)lr_min > 0.f))
        return fail(MPTRAC_E_INVALID_ARG, "need lr_max >= lr_min > 0 (and lr_min > 0 in float32)");
    const int64_t steps = n / batch;
    if (step0 < 0 || total_steps < 1 || (int64_t)step0 + steps > (int64_t)total_steps)
        return fail(MPTRAC_E_INVALID_ARG, "steps %d .. %lld lie outside the schedule of %d", step0 + 1,
                    (long long)(step0 + steps), total_steps);
    if (!device_accessible(x) || !device_accessible(y) || !device_accessible(loss))
        return fail(MPTRAC_E_INVALID_ARG, "x, y and loss must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double pi = 3.14159265358979323846;
    for (int64_t b = 0; b < steps; ++b) {
        const int step = step0 + 1 + (int)b;
        // cosine decay from lr_max (step 0) to lr_min (step total_steps)
        const double lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + std::cos(pi * (double)step / (double)total_steps));
        MPTRAC_CUDA(surr_forward(s->S, x + b * batch * MPTRAC_SURR_KPAD, batch, st));
        MPTRAC_CUDA(surr_backward(s->S, y + b * batch * MPTRAC_SURR_NOUT, batch, loss, st));
        MPTRAC_CUDA(surr_adam(s->S, (float)lr, step, st));
    }
    return ok();
}

int mptrac_surr_advance(mptrac_ctx* c, mptrac_surr* s, const mptrac_particles* P, double t, double dt_seg,
                        uint8_t* fallback, uint64_t* fallback_count, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    if (s->device != c->device) return fail(MPTRAC_E_INVALID_ARG, "context and surrogate are on different devices");
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (c->nx < 3 || c->ny < 3 || c->nz < 3) return fail(MPTRAC_E_INVALID_ARG, "surrogate needs nx, ny, nz >= 3");
    int s0, s1;
    if ((rc = bracket_slots(c, t, t, s0, s1))) return rc;
    const double t0 = c->t_slot[s0], t1 = c->t_slot[s1];
    if (!(dt_seg > 0)) return fail(MPTRAC_E_INVALID_ARG, "dt_seg must be > 0");
    if (P->n == 0) return ok();
    if (!device_accessible(fallback)) return fail(MPTRAC_E_INVALID_ARG, "fallback must be device memory");
    if (fallback_count && !device_accessible(fallback_count))
        return fail(MPTRAC_E_INVALID_ARG, "fallback_count must be device memory");
    const int window_ok = (t + dt_seg <= t1 + 1e-9 * (t1 - t0)) ? 1 : 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float w = (float)((t - t0) / (t1 - t0));
    MPTRAC_CUDA(launch_surr_fused(c->storage, s->S, c->geo, MetView{c->d_met[s0], c->d_scales[s0]},
                                  MetView{c->d_met[s1], c->d_scales[s1]}, P->n, P->lon, P->lat, P->p, w,
                                  window_ok, fallback, fallback_count, c->lon0, st));
    return ok();
}

int mptrac_surr_set_kernel(mptrac_surr* s, int kernel) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    if (kernel != MPTRAC_SURR_KERNEL_TCGEN05 && kernel != MPTRAC_SURR_KERNEL_MMA_SYNC &&
        kernel != MPTRAC_SURR_KERNEL_WAIT_TEST)
        return fail(MPTRAC_E_INVALID_ARG, "unknown surrogate kernel %d", kernel);
    s->S.kernel = kernel;
    return ok();
}

int mptrac_surr_status(mptrac_surr* s, uintptr_t stream) {
    if (!s) return fail(MPTRAC_E_NOT_INIT, "surrogate is NULL");
    DeviceGuard device_guard_s(s->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int flag = 0;
    MPTRAC_CUDA(cudaMemcpyAsync(&flag, s->S.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPTRAC_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        MPTRAC_CUDA(cudaMemsetAsync(s->S.status, 0, sizeof(int), st));
        MPTRAC_CUDA(cudaStreamSynchronize(st));
        return fail(MPTRAC_E_TIMEOUT, "a bounded wait of the fused surrogate inference gave up");
    }
    return ok();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sorting without any device allocation.
//
// Some callers cannot allocate device memory at all: code that runs while
// another framework owns the device heap (a pool allocator that must not be
// bypassed), code that is not allowed to call cudaMalloc because it would
// synchronise the device in the middle of an asynchronous pipeline, or
// embedded hosts with a fixed memory budget checked at start-up.  For them
// mptrac_sort_noalloc sorts with scratch memory that lives in a file-scope
// device array of fixed size instead of a caller-provided workspace.
//
// The array is part of the library image: every GPU that loads the library
// holds its 16 MiB until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress, with that device current) on the first
// call made on that device; in host code the array's name is only a host-side
// stand-in, never a device address.  No part of the scratch has to start at
// zero: every call writes each scratch byte before it reads it.  All calls on
// a device share the one array, so calls whose work overlaps on the GPU (other
// streams, other threads, other contexts on the same device) race on it and
// must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;
__device__ __align__(256) static unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 128;
std::atomic<void*> g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return fail(MPTRAC_E_CUDA, "no usable CUDA device for the static sort scratch (%s)",
                    e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range");
    }
    void* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return fail(MPTRAC_E_CUDA, "cudaGetSymbolAddress of the static sort scratch failed: %s",
                        cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return MPTRAC_OK;
}

}  // namespace

extern "C" int mptrac_sort_noalloc(mptrac_ctx* c, const mptrac_particles* P, uintptr_t stream) {
    if (!c) return fail(MPTRAC_E_NOT_INIT, "context is NULL");
    DeviceGuard device_guard(c->device);
    int rc = check_particles(P, false);
    if (rc) return rc;
    if (P->n > MPTRAC_SORT_NOALLOC_MAX_N)
        return fail(MPTRAC_E_INVALID_ARG,
                    "mptrac_sort_noalloc sorts at most %d particles (got %lld); use mptrac_sort with a workspace",
                    MPTRAC_SORT_NOALLOC_MAX_N, (long long)P->n);
    if (P->n == 0) return ok();
    if (sort_workspace_bytes(P->n) > kNoallocScratchBytes)
        return fail(MPTRAC_E_WORKSPACE, "static sort scratch too small for %lld particles", (long long)P->n);
    void* ws = nullptr;
    if ((rc = noalloc_scratch(&ws))) return rc;
    MPTRAC_CUDA(run_sort(c->geo, *P, ws, c->key_bits, reinterpret_cast<cudaStream_t>(stream)));
    return ok();
}

