// Particle sorting by met cell (the sorting modules of arxiv 2211.12616,
// Section 6).  key = (j*nx + i)*nz + k of each particle's cell, computed in
// float64 with the same expressions as the interpolation's cell rule, then a
// stable least-significant-digit radix sort of (key, index) pairs with 8-bit
// digits, then one gather of every particle array.
//
// Each pass: (1) per-tile digit histograms, (2) per-digit scan over tiles,
// (3) stable scatter.  A tile is 2048 keys handled by 256 threads in 8 rounds
// of 256 consecutive keys; inside a round, lanes with equal digits find each
// other with __match_any_sync and are ranked by lane, warps are ranked by a
// shared-memory scan, rounds by a running count -- which keeps equal keys in
// their input order.
#include "internal.h"

namespace mptrac {
namespace {

constexpr int kSortThreads = 256;
constexpr int kRounds = 8;
constexpr int kTileKeys = kSortThreads * kRounds;
constexpr int kRadix = 256;

// Cell key from float64 positions, the definition: x = ((lon - lon0) mod 360)
// / dlon, i = floor(x) mod nx; j = floor((lat - lat0) / dlat) clamped to
// [0, ny-2]; k = (number of levels >= clamp(p)) - 1 clamped to [0, nz-2].
__device__ __forceinline__ uint32_t cell_key_f64(double lon, double lat, double p, const Geo& g) {
    double r = fmod(__dsub_rn(lon, g.lon0_d), 360.0);
    if (r < 0.0) r = __dadd_rn(r, 360.0);
    const double x = __ddiv_rn(r, g.dlon_d);
    long long i = (long long)floor(x);
    i %= g.nx;
    if (i < 0) i += g.nx;
    const double y = __ddiv_rn(__dsub_rn(lat, g.lat0_d), g.dlat_d);
    long long j = (long long)floor(y);
    j = j < 0 ? 0 : (j > g.ny - 2 ? g.ny - 2 : j);
    const double pc = fmin(fmax(p, g.pmin_d), g.pmax_d);
    int lo = 0, hi = g.nz;   // plev decreasing: length of the prefix with plev >= pc
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (g.plev_d[mid] >= pc) lo = mid + 1; else hi = mid;
    }
    int k = lo - 1;
    k = k < 0 ? 0 : (k > g.nz - 2 ? g.nz - 2 : k);
    return (uint32_t)((j * g.nx + i) * g.nz + k);
}

struct KeyTables {
    float plev[kMaxNZ];
    int16_t kguess[kGuessBins];
};

// Same key, computed in float32 when that is provably identical: the float32
// cell coordinates are within key_mx / key_my cells (a bound derived from the
// grid on the host, with a factor 8 to spare) and p within ~1e-7 relative of
// the exact values, so estimates farther than that from every cell face
// (and p farther than 1e-5 relative from its bracketing levels) have the same
// floor / level count as the float64 definition.  Anything closer to a face, or outside the regular range, takes
// the float64 path.
__device__ __forceinline__ uint32_t cell_key(double lon, double lat, double p, const Geo& g,
                                             const KeyTables& t) {
    const float lf = (float)lon, af = (float)lat, pf = (float)p;
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
    int k = t.kguess[b];
    while (k > 0 && t.plev[k] < pc) --k;
    while (k < g.nz - 2 && t.plev[k + 1] >= pc) ++k;
    const bool below_top = pf > g.pmax * (1.f + 1e-5f);     // clamps to level 0
    const bool above_bot = pf < g.pmin * (1.f - 1e-5f);     // clamps to the top level
    if (!below_top && !above_bot) {
        const float margin = 1e-5f * pc;
        ok = ok && (t.plev[k] - pc > margin || k == 0) && (pc - t.plev[k + 1] > margin || k == g.nz - 2);
        if (k == 0 && !(pc < t.plev[0] - margin)) ok = false;
        if (k == g.nz - 2 && !(pc > t.plev[g.nz - 1] + margin)) ok = false;
    }
    if (!ok || !(lf == lf) || !(af == af) || !(pf == pf)) return cell_key_f64(lon, lat, p, g);
    const int i = (int)xf;
    return (uint32_t)((j * g.nx + i) * g.nz + k);
}

__global__ void k_keys(Geo g, int64_t n, const double* lon, const double* lat, const double* p,
                       uint32_t* keys, uint32_t* vals) {
    __shared__ KeyTables t;
    for (int q = threadIdx.x; q < g.nz; q += blockDim.x) t.plev[q] = g.plev[q];
    for (int q = threadIdx.x; q < g.nbins; q += blockDim.x) t.kguess[q] = g.kguess[q];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        keys[q] = cell_key(lon[q], lat[q], p[q], g, t);
        if (vals) vals[q] = (uint32_t)q;
    }
}

// write_grid: particles per met cell; lanes of a warp with the same cell (common
// once particles are sorted) add their count with one atomic.
__global__ void k_grid_counts(Geo g, int64_t n, const double* lon, const double* lat, const double* p,
                              uint32_t* counts) {
    __shared__ KeyTables tb;
    for (int q = threadIdx.x; q < g.nz; q += blockDim.x) tb.plev[q] = g.plev[q];
    for (int q = threadIdx.x; q < g.nbins; q += blockDim.x) tb.kguess[q] = g.kguess[q];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t span = (n + stride - 1) / stride * stride;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < span; q += stride) {
        const bool valid = q < n;
        const uint32_t key = valid ? cell_key(lon[q], lat[q], p[q], g, tb) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(__activemask(), key);
        const int lane = threadIdx.x & 31;
        if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&counts[key], (uint32_t)__popc(peers));
    }
}

// Cell keys (or the inactive key) of one tile of 2048 particles plus that
// tile's histogram of the lowest 8-bit digit: the first radix pass needs no
// separate histogram launch.
__global__ void __launch_bounds__(kSortThreads) k_keys_hist(Geo g, int64_t n, const double* lon,
                                                            const double* lat, const double* p,
                                                            const uint32_t* release, double t,
                                                            const double* ts, const double* te, int nrel,
                                                            uint32_t inactive_key, uint32_t* keys,
                                                            uint32_t* hist, int ntiles) {
    __shared__ KeyTables tb;
    __shared__ uint32_t h[kRadix];
    for (int q = threadIdx.x; q < g.nz; q += blockDim.x) tb.plev[q] = g.plev[q];
    for (int q = threadIdx.x; q < g.nbins; q += blockDim.x) tb.kguess[q] = g.kguess[q];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileKeys;
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * kSortThreads + threadIdx.x;
        if (q >= n) continue;
        bool active = true;
        if (release) {
            const uint32_t rr = release[q];
            active = rr < (uint32_t)nrel && t >= ts[rr] && t < te[rr];
        }
        const uint32_t k = active ? cell_key(lon[q], lat[q], p[q], g, tb) : inactive_key;
        keys[q] = k;
        atomicAdd(&h[k & 0xFF], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// hist[d * ntiles + tile] = number of keys of `tile` with digit d
__global__ void __launch_bounds__(kSortThreads) k_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                       int shift, uint32_t* hist, int ntiles) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileKeys;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * kSortThreads + threadIdx.x;
        if (q < n) atomicAdd(&h[(keys[q] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of its row of tile counts; row total to tot[d].
__global__ void __launch_bounds__(kSortThreads) k_scan_rows(uint32_t* hist, int ntiles, uint32_t* tot) {
    __shared__ uint32_t warp_sum[kSortThreads / 32];
    __shared__ uint32_t carry;
    uint32_t* row = hist + (int64_t)blockIdx.x * ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += kSortThreads) {
        const int q = base + threadIdx.x;
        const uint32_t v = q < ntiles ? row[q] : 0u;
        uint32_t incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        uint32_t wpre = 0, total = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t s = warp_sum[w];
            if (w < wid) wpre += s;
            total += s;
        }
        const uint32_t c = carry;
        if (q < ntiles) row[q] = c + wpre + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Stable scatter of one tile (2048 keys) for one 8-bit digit.  Warp w owns the
// tile's keys [256 w, 256 w + 256) and walks them in 8 rounds of 32
// consecutive keys: lanes with equal digits find each other with
// __match_any_sync and take ranks from a warp-private running count in shared
// memory.  Scans over warps and over digits then give every key its place in
// the tile sorted by digit (stable); the tile is staged in that order in
// shared memory and written out by consecutive threads, so each digit's run
// of keys lands in consecutive global addresses (coalesced writes).
__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint32_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint32_t* __restrict__ kout,
                                                          uint32_t* __restrict__ vout, int64_t n,
                                                          int shift, const uint32_t* __restrict__ offs,
                                                          const uint32_t* __restrict__ tot, int ntiles) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t s_wc[W][kRadix];
    __shared__ uint32_t s_base[kRadix];   // global start of each digit's run of this tile
    __shared__ uint32_t s_tp[kRadix];     // start of each digit inside the staged tile
    __shared__ uint32_t s_ws[W];
    __shared__ uint32_t s_key[kTileKeys];
    __shared__ uint32_t s_val[kTileKeys];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < kRadix / 32; ++q) s_wc[wid][q * 32 + lane] = 0;
    {   // exclusive scan of the digit totals + this tile's offset within each digit
        const uint32_t v = tot[tid];
        uint32_t incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) s_ws[wid] = incl;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < wid; ++w) pre += s_ws[w];
        s_base[tid] = pre + incl - v + offs[(int64_t)tid * ntiles + blockIdx.x];
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kTileKeys;
    const int64_t base = tile0 + (int64_t)wid * (kRounds * 32);
    uint32_t key[kRounds], val[kRounds], rank[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * 32 + lane;
        const bool valid = q < n;
        key[r] = valid ? kin[q] : 0xFFFFFFFFu;
        val[r] = valid ? (vin ? vin[q] : (uint32_t)q) : 0u;
    }
    __syncthreads();   // every warp's counters zeroed, s_ws reusable
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * 32 + lane;
        const bool valid = q < n;
        const uint32_t d = (key[r] >> shift) & 0xFF;
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : (kRadix + lane));
        rank[r] = valid ? s_wc[wid][d] + __popc(peers & lt_mask) : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) s_wc[wid][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // thread = digit: prefix over warps, then exclusive scan of the tile's digit counts
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = s_wc[w][tid];
            s_wc[w][tid] = run;
            run += c;
        }
        uint32_t incl = run;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) s_ws[wid] = incl;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < wid; ++w) pre += s_ws[w];
        s_tp[tid] = pre + incl - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * 32 + lane;
        if (q < n) {
            const uint32_t d = (key[r] >> shift) & 0xFF;
            const uint32_t loc = s_tp[d] + s_wc[wid][d] + rank[r];
            s_key[loc] = key[r];
            s_val[loc] = val[r];
        }
    }
    __syncthreads();
    const int64_t left = n - tile0;
    const int cnt = left < kTileKeys ? (int)left : kTileKeys;
    for (int e = tid; e < cnt; e += kSortThreads) {
        const uint32_t k = s_key[e];
        const uint32_t d = (k >> shift) & 0xFF;
        const uint32_t pos = s_base[d] + (uint32_t)e - s_tp[d];
        kout[pos] = k;
        vout[pos] = s_val[e];
    }
}

struct PermArgs {
    int64_t n;
    const uint32_t* perm;
    double* dst_d[3];
    const double* src_d[3];
    uint32_t* dst_u[2];
    const uint32_t* src_u[2];
    float* dst_f[3];
    const float* src_f[3];
};

__global__ void k_permute(const __grid_constant__ PermArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t s = a.perm[q];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (a.dst_d[c]) a.dst_d[c][q] = a.src_d[c][s];
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (a.dst_u[c]) a.dst_u[c][q] = a.src_u[c][s];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (a.dst_f[c]) a.dst_f[c][q] = a.src_f[c][s];
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t ntiles_for(int64_t n) { return (n + kTileKeys - 1) / kTileKeys; }

struct WsLayout {
    size_t keys_a, keys_b, vals_a, vals_b, hist, tot, copy_d, copy_u, copy_f, total;
};

WsLayout ws_layout(int64_t n) {
    WsLayout L{};
    size_t o = 0;
    const size_t nn = (size_t)(n > 0 ? n : 0);
    const size_t nt = (size_t)ntiles_for(n);
    L.keys_a = o; o += align256(nn * 4);
    L.keys_b = o; o += align256(nn * 4);
    L.vals_a = o; o += align256(nn * 4);
    L.vals_b = o; o += align256(nn * 4);
    L.hist = o; o += align256(nt * kRadix * 4);
    L.tot = o; o += align256(kRadix * 4);
    L.copy_d = o; o += align256(nn * 8) * 3;
    L.copy_u = o; o += align256(nn * 4) * 2;
    L.copy_f = o; o += align256(nn * 4) * 3;
    L.total = o;
    return L;
}

int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (int)b;
}

}  // namespace

size_t sort_workspace_bytes(int64_t n) { return ws_layout(n).total; }

cudaError_t launch_cell_keys(const Geo& g, int64_t n, const double* lon, const double* lat,
                             const double* p, uint32_t* keys, cudaStream_t s) {
    note_launches(1);
    k_keys<<<grid_for(n), 256, 0, s>>>(g, n, lon, lat, p, keys, nullptr);
    return cudaGetLastError();
}

namespace {

// LSD radix passes over the keys already in the workspace's keys_a, then the
// gather of every particle array in sorted order.
cudaError_t sort_from_keys(const mptrac_particles& P, void* ws, int key_bits, cudaStream_t s,
                           bool first_hist_done = false) {
    const int64_t n = P.n;
    const WsLayout L = ws_layout(n);
    char* w = static_cast<char*>(ws);
    uint32_t* ka = reinterpret_cast<uint32_t*>(w + L.keys_a);
    uint32_t* kb = reinterpret_cast<uint32_t*>(w + L.keys_b);
    uint32_t* va = reinterpret_cast<uint32_t*>(w + L.vals_a);
    uint32_t* vb = reinterpret_cast<uint32_t*>(w + L.vals_b);
    uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
    uint32_t* tot = reinterpret_cast<uint32_t*>(w + L.tot);
    const int ntiles = (int)ntiles_for(n);
    cudaError_t e;
    const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
    note_launches(1 + 3 * passes - (first_hist_done ? 1 : 0));
    bool first = true;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        if (!(pass == 0 && first_hist_done)) k_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, hist, ntiles);
        k_scan_rows<<<kRadix, kSortThreads, 0, s>>>(hist, ntiles, tot);
        k_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, first ? nullptr : va, kb, vb, n, shift, hist,
                                                  tot, ntiles);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        first = false;
        uint32_t* tmp = ka; ka = kb; kb = tmp;
        tmp = va; va = vb; vb = tmp;
    }
    // copy the arrays aside, then gather them back in sorted order
    PermArgs pa{};
    pa.n = n;
    pa.perm = va;
    double* dd[3] = {P.lon, P.lat, P.p};
    uint32_t* uu[2] = {P.id, P.release};
    float* fl[3] = {P.up, P.vp, P.wp};
    for (int c = 0; c < 3; ++c) {
        if (!dd[c]) continue;
        double* cp = reinterpret_cast<double*>(w + L.copy_d + c * align256((size_t)n * 8));
        if ((e = cudaMemcpyAsync(cp, dd[c], (size_t)n * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        pa.dst_d[c] = dd[c];
        pa.src_d[c] = cp;
    }
    for (int c = 0; c < 2; ++c) {
        if (!uu[c]) continue;
        uint32_t* cp = reinterpret_cast<uint32_t*>(w + L.copy_u + c * align256((size_t)n * 4));
        if ((e = cudaMemcpyAsync(cp, uu[c], (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        pa.dst_u[c] = uu[c];
        pa.src_u[c] = cp;
    }
    for (int c = 0; c < 3; ++c) {
        if (!fl[c]) continue;
        float* cp = reinterpret_cast<float*>(w + L.copy_f + c * align256((size_t)n * 4));
        if ((e = cudaMemcpyAsync(cp, fl[c], (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        pa.dst_f[c] = fl[c];
        pa.src_f[c] = cp;
    }
    k_permute<<<grid_for(n), 256, 0, s>>>(pa);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grid_counts(const Geo& g, int64_t n, const double* lon, const double* lat,
                               const double* p, uint32_t* counts, cudaStream_t s) {
    note_launches(1);
    k_grid_counts<<<grid_for(n), 256, 0, s>>>(g, n, lon, lat, p, counts);
    return cudaGetLastError();
}

cudaError_t run_sort(const Geo& g, const mptrac_particles& P, void* ws, int key_bits,
                     cudaStream_t s) {
    const int64_t n = P.n;
    if (n <= 0) return cudaSuccess;
    const WsLayout L = ws_layout(n);
    uint32_t* ka = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.keys_a);
    uint32_t* hist = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.hist);
    const int ntiles = (int)ntiles_for(n);
    note_launches(1);
    k_keys_hist<<<ntiles, kSortThreads, 0, s>>>(g, n, P.lon, P.lat, P.p, nullptr, 0.0, nullptr, nullptr, 0, 0u,
                                                ka, hist, ntiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sort_from_keys(P, ws, key_bits, s, true);
}

cudaError_t run_sort_at(const Geo& g, const mptrac_particles& P, void* ws, int key_bits, double t,
                        const double* ts, const double* te, int nrel, cudaStream_t s) {
    const int64_t n = P.n;
    if (n <= 0) return cudaSuccess;
    const WsLayout L = ws_layout(n);
    uint32_t* ka = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.keys_a);
    uint32_t* hist = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.hist);
    const int ntiles = (int)ntiles_for(n);
    note_launches(1);
    k_keys_hist<<<ntiles, kSortThreads, 0, s>>>(g, n, P.lon, P.lat, P.p, P.release, t, ts, te, nrel,
                                                1u << key_bits, ka, hist, ntiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sort_from_keys(P, ws, key_bits + 1, s, true);
}

}  // namespace mptrac
