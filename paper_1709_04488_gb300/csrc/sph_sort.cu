// Morton keys and a stable LSD radix sort of (key, index) pairs.
//
// The paper builds a KD tree by recursive median bisection (Sec. 4.2, tree;
// Sec. 5.2 notes the serial top levels limit its parallel scaling).  Here the
// spatial order comes from one fully parallel sort instead: a 30-bit Morton
// key (10 bits per axis) per particle, prefixed by the problem index in a
// batch, sorted stably so that ties keep the original particle order.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kSortThreads = 256;
// keys per thread of a radix pass (1, 2, 4 or 8): small problems take short
// tiles (more blocks in flight), large ones long tiles (fewer look-back records)
#ifndef SPH_SORT_ITEMS_S
#define SPH_SORT_ITEMS_S 2  // up to 2^18 keys
#endif
#ifndef SPH_SORT_ITEMS_M
#define SPH_SORT_ITEMS_M 8  // up to 2^22 keys
#endif
#ifndef SPH_SORT_ITEMS_L
#define SPH_SORT_ITEMS_L 8
#endif
int sort_items(long long n)
{
    return n <= (1ll << 18) ? SPH_SORT_ITEMS_S : n <= (1ll << 22) ? SPH_SORT_ITEMS_M : SPH_SORT_ITEMS_L;
}
constexpr int kBboxThreads = 1024, kBboxItems = 64;

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Shared-memory histogram update aggregated over the warp: lanes holding the
// same digit are combined first (Morton digits of neighbouring keys repeat,
// and 32 atomics on one address would serialise).  Every lane of the warp
// must call it; lanes with valid == false contribute nothing.
__device__ __forceinline__ void warp_hist_add(unsigned *h, unsigned d, bool valid)
{
    const int lane = threadIdx.x & 31;
    unsigned dd = valid ? d : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, dd);
    if (valid && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&h[d], (unsigned)__popc(peers));
}

__global__ void k_reset_bbox(ProbDyn *dyn, int nprob)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    for (int a = 0; a < 3; ++a) {
        dyn[p].bbox_bits[a] = ~0ull;   // running minimum
        dyn[p].bbox_bits[3 + a] = 0ull; // running maximum
    }
}

// Bounding box of isolated problems (FP64, ordered-integer atomics).  Each
// block takes items * blockDim consecutive particles, kept per problem in
// registers; a block within one problem reduces over the block (one set of
// atomics per block), else each thread adds its own on a change of problem.
__device__ __forceinline__ void bbox_flush(const BatchView &b, int p, const unsigned long long *v)
{
    if (v[0] == ~0ull) return;  // nothing of an isolated problem seen
    for (int a = 0; a < 3; ++a) {
        atomicMin(&b.dyn[p].bbox_bits[a], v[a]);
        atomicMax(&b.dyn[p].bbox_bits[3 + a], v[3 + a]);
    }
}

__global__ void k_bbox(BatchView b, int items)
{
    __shared__ unsigned long long red[6][kBboxThreads / 32];
    __shared__ int pfirst, plast;
    const long long base = (long long)blockIdx.x * blockDim.x * items;
    if (base >= b.ntot) return;
    const long long end = base + (long long)blockDim.x * items < b.ntot ? base + (long long)blockDim.x * items : b.ntot;
    if (threadIdx.x == 0) {
        pfirst = find_problem(b.prob_base, b.nprob, base);
        plast = find_problem(b.prob_base, b.nprob, end - 1);
    }
    __syncthreads();
    unsigned long long v[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
    int cur = -1;
    for (long long g = base + threadIdx.x; g < end; g += blockDim.x) {
        const int p = pfirst == plast ? pfirst : find_problem(b.prob_base, b.nprob, g);
        if (p != cur) {
            if (cur >= 0) bbox_flush(b, cur, v);
            for (int a = 0; a < 3; ++a) {
                v[a] = ~0ull;
                v[3 + a] = 0ull;
            }
            cur = p;
        }
        const ProbStatic &ps = b.prob[p];
        if (ps.ph.periodic) continue;  // (periodic boxes need no pass)
        const long long i = g - ps.base;
        const unsigned long long X[3] = {ordered_bits(ps.x[i]), ordered_bits(ps.y[i]), ordered_bits(ps.z[i])};
        for (int a = 0; a < 3; ++a) {
            v[a] = X[a] < v[a] ? X[a] : v[a];
            v[3 + a] = X[a] > v[3 + a] ? X[a] : v[3 + a];
        }
    }
    if (pfirst != plast) {
        if (cur >= 0) bbox_flush(b, cur, v);
        return;
    }
    for (int a = 0; a < 6; ++a) {
        unsigned long long x = v[a];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
            x = a < 3 ? (y < x ? y : x) : (y > x ? y : x);
        }
        if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        unsigned long long w[6];
        for (int a = 0; a < 6; ++a) {
            unsigned long long x = threadIdx.x < nw ? red[a][threadIdx.x] : (a < 3 ? ~0ull : 0ull);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                x = a < 3 ? (y < x ? y : x) : (y > x ? y : x);
            }
            w[a] = x;
        }
        if (threadIdx.x == 0) bbox_flush(b, pfirst, w);
    }
}

__global__ void k_domain(BatchView b)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.nprob) return;
    const PhysParams &ph = b.prob[p].ph;
    ProbDyn &d = b.dyn[p];
    double ext = 0.0;
    if (ph.periodic) {
        for (int a = 0; a < 3; ++a) {
            d.dom_lo[a] = ph.box_lo[a];
            ext = fmax(ext, ph.box_len[a]);
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            double lo = from_ordered_bits(d.bbox_bits[a]);
            double hi = from_ordered_bits(d.bbox_bits[3 + a]);
            if (b.prob[p].n == 0) lo = hi = 0.0;
            d.dom_lo[a] = lo;
            ext = fmax(ext, hi - lo);
        }
        ext = ext * (1.0 + 1e-9) + 1e-300;
    }
    d.dom_inv = ext > 0.0 ? 1.0 / ext : 1.0;
}

// ---- single-pass LSD radix sort ("onesweep"): one fused key + histogram
// kernel for all passes, then one kernel per 8-bit pass whose tiles find
// their global offsets by a decoupled look-back over the earlier tiles.
constexpr unsigned kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kCountMask = (1u << 30) - 1u;
constexpr long long kSpinLimit = 1ll << 24;
constexpr int kLookBack = 8;

__device__ __forceinline__ unsigned morton_key_code(const BatchView &b, int p, long long g)
{
    const ProbStatic &ps = b.prob[p];
    const ProbDyn &d = b.dyn[p];
    long long i = g - ps.base;
    double X[3] = {ps.x[i], ps.y[i], ps.z[i]};
    double lo[3], inv;
    if (ps.ph.periodic) {
        double ext = fmax(ps.ph.box_len[0], fmax(ps.ph.box_len[1], ps.ph.box_len[2]));
        for (int a = 0; a < 3; ++a) lo[a] = ps.ph.box_lo[a];
        inv = 1.0 / ext;
    } else {
        for (int a = 0; a < 3; ++a) lo[a] = d.dom_lo[a];
        inv = d.dom_inv;
    }
    unsigned code = 0;
    for (int a = 0; a < 3; ++a) {
        double t = (X[a] - lo[a]) * inv * (double)(1 << kMortonBits);
        int c = t > 0.0 ? (int)t : 0;  // NaN maps to 0
        c = c > (1 << kMortonBits) - 1 ? (1 << kMortonBits) - 1 : c;
        code |= spread10((unsigned)c) << a;
    }
    return code;
}

// Keys of every particle, and the digit histograms of every pass.
__global__ void k_keys_hist(BatchView b, unsigned long long *kout, unsigned *hist, int passes, int lo)
{
    __shared__ unsigned h[8][256];
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) (&h[0][0])[k] = 0u;
    __syncthreads();
    for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < b.ntot; g0 += (long long)gridDim.x * blockDim.x) {
        const long long g = g0 + threadIdx.x;
        const bool ok = g < b.ntot;
        unsigned long long key = 0ull;
        if (ok) {
            int p = find_problem(b.prob_base, b.nprob, g);
            key = ((unsigned long long)p << kMortonTotal) | (morton_key_code(b, p, g) & ~((1u << lo) - 1u));
            kout[g] = key;
        }
        for (int q = 0; q < passes; ++q) warp_hist_add(h[q], (unsigned)(key >> (lo + 8 * q)) & 255u, ok);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * 256; k += blockDim.x) {
        unsigned v = (&h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

template <int ITEMS>
__global__ void k_onesweep(const unsigned long long *kin, const unsigned *vin, unsigned long long *kout,
                           unsigned *vout, long long n, int shift, const unsigned *hist, unsigned *status,
                           unsigned *tile_ctr, int identity_vals, unsigned *timeout_flag)
{
    constexpr int NW = kSortThreads / 32;
    constexpr int TILE = kSortThreads * ITEMS;
    __shared__ unsigned run[256];
    __shared__ unsigned wcnt[NW][256];
    __shared__ unsigned cnt[256];
    __shared__ unsigned gpre[256];
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = threadIdx.x;
    if (t == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    cnt[t] = 0u;
    for (int w = 0; w < NW; ++w) wcnt[w][t] = 0u;
    // exclusive scan of the pass's global digit histogram
    gpre[t] = hist[t];
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        unsigned v = t >= o ? gpre[t - o] : 0u;
        __syncthreads();
        gpre[t] += v;
        __syncthreads();
    }
    const unsigned gstart = gpre[t] - hist[t];
    const int tile = s_tile;
    const long long base = (long long)tile * TILE;
    // local digit counts
    unsigned long long keys[ITEMS];
    for (int r = 0; r < ITEMS; ++r) {
        long long k = base + r * kSortThreads + t;
        keys[r] = k < n ? kin[k] : 0ull;
        warp_hist_add(cnt, (unsigned)(keys[r] >> shift) & 255u, k < n);
    }
    __syncthreads();
    // publish this tile's counts, then look back over the earlier tiles
    unsigned *st = status + (long long)tile * 256;
    const unsigned mine = cnt[t];
    if (tile == 0) {
        atomicExch(&st[t], kFlagPre | mine);
        run[t] = gstart;
    } else {
        atomicExch(&st[t], kFlagAgg | mine);
        // look back over the earlier tiles' counts of digit t, kLookBack
        // predecessors per round (their loads in flight together)
        unsigned excl = 0u;
        long long spins = 0;
        for (int pred = tile - 1; pred >= 0;) {
            unsigned v[kLookBack];
#pragma unroll
            for (int k = 0; k < kLookBack; ++k)
                v[k] = pred - k >= 0 ? (unsigned)*(volatile unsigned *)(status + (long long)(pred - k) * 256 + t) : (unsigned)kFlagPre;
            int used = 0;
            bool done = false, pending = false;
#pragma unroll
            for (int k = 0; k < kLookBack; ++k) {
                if (done || pending) continue;
                const unsigned f = v[k] & ~kCountMask;
                if (f == 0u) {
                    pending = true;
                    continue;
                }
                excl += v[k] & kCountMask;
                ++used;
                if (f == kFlagPre) done = true;
            }
            if (done) break;
            pred -= used;
            if (pending && ++spins > kSpinLimit) {
                atomicOr(timeout_flag, 1u);
                break;
            }
        }
        atomicExch(&st[t], kFlagPre | (excl + mine));
        run[t] = gstart + excl;
    }
    __syncthreads();
    // stable ranks inside the tile (index order), then scatter
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < ITEMS; ++r) {
        long long k = base + r * kSortThreads + t;
        bool ok = k < n;
        unsigned long long key = keys[r];
        unsigned val = ok ? (identity_vals ? (unsigned)k : vin[k]) : 0u;
        unsigned d = ok ? (unsigned)(key >> shift) & 255u : 256u + lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        bool leader = (peers & lt) == 0u;
        if (ok && leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            unsigned off = run[d] + rank;
            for (int w = 0; w < warp; ++w) off += wcnt[w][d];
            kout[off] = key;
            vout[off] = val;
        }
        __syncthreads();
        unsigned tot = 0;
        for (int w = 0; w < NW; ++w) {
            tot += wcnt[w][t];
            wcnt[w][t] = 0;
        }
        run[t] += tot;
        __syncthreads();
    }
}


}  // namespace

cudaError_t launch_domain_and_keys(const BatchView &b, cudaStream_t st)
{
    // the keys themselves are formed by the sort's first kernel; here only the
    // bounding boxes of isolated problems (periodic boxes need no pass)
    if (b.ntot == 0 || !b.any_isolated) return cudaSuccess;
    int pb = (b.nprob + 127) / 128;
    k_reset_bbox<<<pb, 128, 0, st>>>(b.dyn, b.nprob);
    // two blocks per SM of up to kBboxItems particles a thread
    const long long fill = 2LL * dev_info().sm_count * kBboxThreads;
    long long items = (b.ntot + fill - 1) / fill;
    items = items < 1 ? 1 : items > kBboxItems ? kBboxItems : items;
    const long long nb = (b.ntot + kBboxThreads * items - 1) / (kBboxThreads * items);
    k_bbox<<<(unsigned)nb, kBboxThreads, 0, st>>>(b, (int)items);
    k_domain<<<pb, 128, 0, st>>>(b);
    return cudaGetLastError();
}

long long sort_tiles(long long n)
{
    const long long t = (long long)kSortThreads * sort_items(n);
    return (n + t - 1) / t;
}

cudaError_t launch_radix_sort(const BatchView &b, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    const long long n = b.ntot;
    const int items = sort_items(n);
    const long long tile_keys = (long long)kSortThreads * items;
    const int ntile = (int)((n + tile_keys - 1) / tile_keys);
    const int passes = (b.key_bits - b.key_lo + 7) / 8;
    // hist[passes][256] | tile counters[passes] | status[passes][ntile][256]
    unsigned *hist = b.hist, *ctr = b.hist + passes * 256, *status = b.hist + passes * 256 + 8;
    cudaMemsetAsync(b.hist, 0, sizeof(unsigned) * ((size_t)passes * 256 + 8 + (size_t)passes * ntile * 256), st);
    int kb = (int)((n + 255) / 256);
    int cap = dev_info().sm_count * 8;
    // the passes ping-pong between the two key buffers: start in the one that
    // leaves the sorted keys in keys[0] for the leaf builder
    int src = passes & 1;
    k_keys_hist<<<kb < cap ? kb : cap, 256, 0, st>>>(b, b.keys[src], hist, passes, b.key_lo);
    for (int pass = 0; pass < passes; ++pass) {
        const bool last = pass == passes - 1;
        unsigned *vdst = last ? (unsigned *)b.perm : b.vals[src ^ 1];
        auto kern = items == 1 ? k_onesweep<1> : items == 2 ? k_onesweep<2> : items == 4 ? k_onesweep<4> : k_onesweep<8>;
        kern<<<ntile, kSortThreads, 0, st>>>(b.keys[src], b.vals[src], b.keys[src ^ 1], vdst, n, b.key_lo + 8 * pass,
                                             hist + pass * 256, status + (size_t)pass * ntile * 256, ctr + pass,
                                             pass == 0, (unsigned *)&b.counters[kTimeoutCounter]);
        src ^= 1;
    }
    return cudaGetLastError();
}

}  // namespace sph
