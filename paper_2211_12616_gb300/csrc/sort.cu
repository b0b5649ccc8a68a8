// Particle sorting by met cell (the sorting modules of arxiv 2211.12616,
// Section 6).  key = (j*nx + i)*nz + k of each particle's cell, computed in
// float64 with the same expressions as the interpolation's cell rule, then a
// stable least-significant-digit radix sort of (key, index) pairs with 8-bit
// digits.  The key kernel also copies every particle array aside, and the
// last pass gathers them from there into their sorted places.
//
// Each pass: (1) per-tile digit histograms, (2) per-digit scan over tiles,
// (3) stable scatter.  A tile is 1024 keys handled by 256 threads in 4 rounds
// of 256 consecutive keys (about 6 tiles per SM for 1e6 particles); inside a round, lanes with equal digits find each
// other with __match_any_sync and are ranked by lane, warps are ranked by a
// shared-memory scan, rounds by a running count -- which keeps equal keys in
// their input order.
#include "cell_key.cuh"
#include "internal.h"

namespace mptrac {
namespace {

constexpr int kSortThreads = 256;
constexpr int kRounds = 4;
constexpr int kTileKeys = kSortThreads * kRounds;
constexpr int kRadix = kSortRadix;
static_assert(kTileKeys == kSortTileKeys, "tile size shared with the fused step");

__global__ void k_keys(Geo g, int64_t n, const double* lon, const double* lat, const double* p,
                       uint32_t* keys, uint32_t* vals) {
    __shared__ KeyTables t;
    load_key_tables(t, g);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        keys[q] = cell_key(lon[q], lat[q], p[q], g, t.plev, t.kguess, t.plev_d);
        if (vals) vals[q] = (uint32_t)q;
    }
}

// write_grid: particles per met cell; lanes of a warp with the same cell (common
// once particles are sorted) add their count with one atomic.
__global__ void k_grid_counts(Geo g, int64_t n, const double* lon, const double* lat, const double* p,
                              uint32_t* counts) {
    __shared__ KeyTables tb;
    load_key_tables(tb, g);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t span = (n + stride - 1) / stride * stride;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < span; q += stride) {
        const bool valid = q < n;
        const uint32_t key = valid ? cell_key(lon[q], lat[q], p[q], g, tb.plev, tb.kguess, tb.plev_d) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(__activemask(), key);
        const int lane = threadIdx.x & 31;
        if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&counts[key], (uint32_t)__popc(peers));
    }
}

// Adds the warp's valid digits to the shared histogram h: lanes with equal
// digits (most of a warp of cell keys once the particles are sorted) are
// counted by one atomic of their lowest lane.  Called by every lane of the
// warp.  (After the first pass equal digits are rare within a warp, and the
// plain atomics of k_hist are cheaper.)
__device__ __forceinline__ void hist_add(uint32_t* h, bool valid, uint32_t digit) {
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 0x100u);
    const int lane = threadIdx.x & 31;
    if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&h[digit], (uint32_t)__popc(peers));
}

struct KeysArgs {
    Geo g;
    int64_t n;
    Arrays part, copy;
    double t;                      // time of the activity test (release windows)
    const double *ts, *te;         // release windows [ts, te), or null: all active
    int nrel;
    uint32_t inactive_key;
    uint32_t* keys;
    uint32_t* hist;
    int ntiles;
};

// Cell keys (or the inactive key) of one tile of particles plus that
// tile's histogram of the lowest 8-bit digit: the first radix pass needs no
// separate histogram launch.  Every particle array is copied aside on the way.
__global__ void __launch_bounds__(kSortThreads) k_keys_hist(const __grid_constant__ KeysArgs a) {
    __shared__ KeyTables tb;
    __shared__ uint32_t h[kRadix];
    const Geo& g = a.g;
    load_key_tables(tb, g);
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileKeys + threadIdx.x;
    // every load of the thread's kRounds particles first (the copies may not be
    // written before them: the compiler cannot tell the arrays apart)
    double vd[kRounds][3];
    uint32_t vu[kRounds][2];
    float vf[kRounds][3];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * kSortThreads;
        if (q >= a.n) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) vd[r][c] = a.part.d[c][q];
#pragma unroll
        for (int c = 0; c < 2; ++c) vu[r][c] = a.part.u[c] ? a.part.u[c][q] : 0u;
#pragma unroll
        for (int c = 0; c < 3; ++c) vf[r][c] = a.part.f[c] ? a.part.f[c][q] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * kSortThreads;
        if (q >= a.n) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) a.copy.d[c][q] = vd[r][c];
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (a.part.u[c]) a.copy.u[c][q] = vu[r][c];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (a.part.f[c]) a.copy.f[c][q] = vf[r][c];
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t q = base + r * kSortThreads;
        const bool valid = q < a.n;
        uint32_t k = 0;
        if (valid) {
            bool active = true;
            if (a.part.u[1] && a.ts) {
                const uint32_t rr = vu[r][1];
                active = rr < (uint32_t)a.nrel && a.t >= a.ts[rr] && a.t < a.te[rr];
            }
            k = active ? cell_key(vd[r][0], vd[r][1], vd[r][2], g, tb.plev, tb.kguess, tb.plev_d) : a.inactive_key;
            a.keys[q] = k;
        }
        hist_add(h, valid, k & 0xFF);
    }
    __syncthreads();
    a.hist[(int64_t)threadIdx.x * a.ntiles + blockIdx.x] = h[threadIdx.x];
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

// Stable scatter of one tile (kTileKeys keys) for one 8-bit digit.  Warp w owns
// the tile's keys [32 kRounds w, 32 kRounds (w + 1)) and walks them in kRounds rounds of 32
// consecutive keys: lanes with equal digits find each other with
// __match_any_sync and take ranks from a warp-private running count in shared
// memory.  Scans over warps and over digits then give every key its place in
// the tile sorted by digit (stable); the tile is staged in that order in
// shared memory and written out by consecutive threads, so each digit's run
// of keys lands in consecutive global addresses (coalesced writes).  In the
// last pass (FINAL) the keys and indices are not written: each sorted place
// receives the particle's values, gathered from the copies.
template <bool FINAL>
__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint32_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint32_t* __restrict__ kout,
                                                          uint32_t* __restrict__ vout, int64_t n,
                                                          int shift, const uint32_t* __restrict__ offs,
                                                          const uint32_t* __restrict__ tot, int ntiles,
                                                          const __grid_constant__ Arrays part,
                                                          const __grid_constant__ Arrays copy) {
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
    if (FINAL) {
        // gather every value of the thread's kRounds places first, then store
        // (the particle arrays and their copies cannot be told apart by the compiler)
        double vd[kRounds][3];
        uint32_t vu[kRounds][2];
        float vf[kRounds][3];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int e = tid + r * kSortThreads;
            if (e >= cnt) continue;
            const uint32_t src = s_val[e];
#pragma unroll
            for (int c = 0; c < 3; ++c) vd[r][c] = copy.d[c][src];
#pragma unroll
            for (int c = 0; c < 2; ++c) vu[r][c] = part.u[c] ? copy.u[c][src] : 0u;
#pragma unroll
            for (int c = 0; c < 3; ++c) vf[r][c] = part.f[c] ? copy.f[c][src] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int e = tid + r * kSortThreads;
            if (e >= cnt) continue;
            const uint32_t d = (s_key[e] >> shift) & 0xFF;
            const uint32_t pos = s_base[d] + (uint32_t)e - s_tp[d];
#pragma unroll
            for (int c = 0; c < 3; ++c) part.d[c][pos] = vd[r][c];
#pragma unroll
            for (int c = 0; c < 2; ++c)
                if (part.u[c]) part.u[c][pos] = vu[r][c];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (part.f[c]) part.f[c][pos] = vf[r][c];
        }
    } else {
        for (int e = tid; e < cnt; e += kSortThreads) {
            const uint32_t k = s_key[e];
            const uint32_t d = (k >> shift) & 0xFF;
            const uint32_t pos = s_base[d] + (uint32_t)e - s_tp[d];
            kout[pos] = k;
            vout[pos] = s_val[e];
        }
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

}  // namespace

size_t sort_workspace_bytes(int64_t n) { return ws_layout(n).total; }

cudaError_t launch_cell_keys(const Geo& g, int64_t n, const double* lon, const double* lat,
                             const double* p, uint32_t* keys, cudaStream_t s) {
    note_launches(1);
    k_keys<<<strided_grid(n, 256, 8), 256, 0, s>>>(g, n, lon, lat, p, keys, nullptr);
    return cudaGetLastError();
}

namespace {

Arrays part_arrays(const mptrac_particles& P) {
    return Arrays{{P.lon, P.lat, P.p}, {P.id, P.release}, {P.up, P.vp, P.wp}};
}

// Workspace copies of the arrays present in P (null where P has none).
Arrays copy_arrays(const mptrac_particles& P, void* ws) {
    const WsLayout L = ws_layout(P.n);
    char* w = static_cast<char*>(ws);
    const size_t n = (size_t)P.n;
    Arrays c{};
    for (int q = 0; q < 3; ++q) c.d[q] = reinterpret_cast<double*>(w + L.copy_d + q * align256(n * 8));
    if (P.id) c.u[0] = reinterpret_cast<uint32_t*>(w + L.copy_u);
    if (P.release) c.u[1] = reinterpret_cast<uint32_t*>(w + L.copy_u + align256(n * 4));
    float* fl[3] = {P.up, P.vp, P.wp};
    for (int q = 0; q < 3; ++q)
        if (fl[q]) c.f[q] = reinterpret_cast<float*>(w + L.copy_f + q * align256(n * 4));
    return c;
}

// Keys, first-digit histograms and copies of the particle arrays (one launch).
cudaError_t keys_and_copies(const Geo& g, const mptrac_particles& P, void* ws, double t, const double* ts,
                            const double* te, int nrel, uint32_t inactive_key, cudaStream_t s) {
    const WsLayout L = ws_layout(P.n);
    KeysArgs a{};
    a.g = g;
    a.n = P.n;
    a.part = part_arrays(P);
    a.copy = copy_arrays(P, ws);
    a.t = t;
    a.ts = ts;
    a.te = te;
    a.nrel = nrel;
    a.inactive_key = inactive_key;
    a.keys = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.keys_a);
    a.hist = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.hist);
    a.ntiles = (int)ntiles_for(P.n);
    note_launches(1);
    k_keys_hist<<<a.ntiles, kSortThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// LSD radix passes over the keys in the workspace's keys_a (first-digit
// histograms already there); the last pass gathers the particle arrays.
cudaError_t sort_from_keys(const mptrac_particles& P, void* ws, int key_bits, cudaStream_t s) {
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
    const Arrays part = part_arrays(P), copy = copy_arrays(P, ws);
    const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
    note_launches(3 * passes - 1);
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        if (pass > 0) k_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, hist, ntiles);
        k_scan_rows<<<kRadix, kSortThreads, 0, s>>>(hist, ntiles, tot);
        const uint32_t* vin = pass == 0 ? nullptr : va;
        if (pass + 1 == passes)
            k_scatter<true><<<ntiles, kSortThreads, 0, s>>>(ka, vin, nullptr, nullptr, n, shift, hist, tot,
                                                            ntiles, part, copy);
        else
            k_scatter<false><<<ntiles, kSortThreads, 0, s>>>(ka, vin, kb, vb, n, shift, hist, tot, ntiles,
                                                             part, copy);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t* tmp = ka; ka = kb; kb = tmp;
        tmp = va; va = vb; vb = tmp;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_grid_counts(const Geo& g, int64_t n, const double* lon, const double* lat,
                               const double* p, uint32_t* counts, cudaStream_t s) {
    note_launches(1);
    k_grid_counts<<<strided_grid(n, 256, 8), 256, 0, s>>>(g, n, lon, lat, p, counts);
    return cudaGetLastError();
}

cudaError_t sort_emit_args(const mptrac_particles& P, void* ws, SortEmit& out, cudaStream_t s) {
    const WsLayout L = ws_layout(P.n);
    out.copy = copy_arrays(P, ws);
    out.keys = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.keys_a);
    out.hist = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.hist);
    out.ntiles = (int)ntiles_for(P.n);
    return cudaMemsetAsync(out.hist, 0, (size_t)out.ntiles * kRadix * sizeof(uint32_t), s);
}

cudaError_t sort_after_emit(const mptrac_particles& P, void* ws, int key_bits, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    return sort_from_keys(P, ws, key_bits, s);
}

cudaError_t run_sort(const Geo& g, const mptrac_particles& P, void* ws, int key_bits,
                     cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    cudaError_t e = keys_and_copies(g, P, ws, 0.0, nullptr, nullptr, 0, 0u, s);
    if (e != cudaSuccess) return e;
    return sort_from_keys(P, ws, key_bits, s);
}

cudaError_t run_sort_at(const Geo& g, const mptrac_particles& P, void* ws, int key_bits, double t,
                        const double* ts, const double* te, int nrel, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    // without a release table every particle is active (ts == null)
    cudaError_t e = keys_and_copies(g, P, ws, t, P.release ? ts : nullptr, te, nrel, 1u << key_bits, s);
    if (e != cudaSuccess) return e;
    return sort_from_keys(P, ws, key_bits + 1, s);
}

}  // namespace mptrac
