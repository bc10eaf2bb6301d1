// Leaf cells and the tree over them (Sec. 4.2, tree; Sec. 4.2 also the
// per-leaf neighbour walk).  The paper's KD tree with N_LEAF-particle leaves
// and per-cell "smallest box containing all the smoothing spheres" is
// replaced by:
//   - leaves = octree cells of the Morton order: for each particle the
//     coarsest cell holding at most 4*leaf_size particles of its problem,
//     split into ceil(count/leaf_size) equal consecutive chunks;
//   - an implicit 32-ary tree over each problem's leaves (32 consecutive
//     leaves per level-1 node, 32 level-1 nodes per level-2 node, ...), whose
//     nodes keep a position box and a smoothing-sphere box, both FP32 rounded
//     outwards from FP64 data.  Node boxes are formed bottom-up in the same
//     kernel as the leaf boxes: the warp that completes a node's last child
//     forms the node.
#include "sph_internal.cuh"
#include "sph_leaf.cuh"

namespace sph {

namespace {

constexpr int kLeafThreads = 256;
constexpr int kLeafItems = 1;  // consecutive particles per thread
constexpr int kLeafTile = kLeafThreads * kLeafItems;
// leaf cell: the coarsest cell with at most cell_limit(leaf size) particles
__host__ __device__ constexpr int cell_limit(int leaf) { return 4 * leaf; }
constexpr int kHalo = 128;  // >= cell_limit of every leaf size (1..32)
constexpr unsigned kTileAgg = 1u << 30, kTilePre = 2u << 30, kTileMask = (1u << 30) - 1u;
constexpr long long kTileSpinLimit = 1ll << 24;

__global__ void k_gather(BatchView b)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.ntot) return;
    int p = (int)(b.keys[0][s] >> kMortonTotal);
    const ProbStatic &ps = b.prob[p];
    long long i = (long long)b.perm[s] - ps.base;
    b.sx[s] = ps.x[i];
    b.sy[s] = ps.y[i];
    b.sz[s] = ps.z[i];
    b.sm[s] = ps.uniform_m ? ps.m_uniform : ps.m[i];  // (equal masses: no random read)
    b.sh[s] = ps.h[i];
}

__device__ __forceinline__ int common_levels(unsigned long long a, unsigned long long b)
{
    unsigned x = (unsigned)((a ^ b) & ((1ull << kMortonTotal) - 1ull));
    if (x == 0u) return kMortonBits;
    return (__clz(x) - (32 - kMortonTotal)) / 3;
}

// Leaf start flag of sorted particle s (see the file comment for the rule);
// K holds the keys of [k0, k0 + kLeafTile + 2 kHalo), s inside the middle part.
// The common key prefix with s shrinks monotonically away from s, so the
// cell of s at level l is found by two binary searches; only levels whose
// cell excludes s - ncell and s + ncell can hold at most ncell particles.
__device__ unsigned leaf_flag(const BatchView &b, const unsigned long long *K, long long k0, long long s)
{
    const unsigned long long ks = K[s - k0];
    const int p = (int)(ks >> kMortonTotal);
    const long long lo = b.prob[p].base, hi = lo + b.prob[p].n - 1;
    const int leaf = kBranch / b.prob[p].lpp, ncell = cell_limit(leaf);
    auto cl = [&](long long t) { return common_levels(ks, K[t - k0]); };
    int l = 0;
    if (s - ncell >= lo) l = max(l, cl(s - ncell) + 1);
    if (s + ncell <= hi) l = max(l, cl(s + ncell) + 1);
    const long long wl = max(lo, s - ncell + 1), wr = min(hi, s + ncell - 1);
    for (; l <= kMortonBits; ++l) {
        long long a = wl, z = s;  // first t with cl(t) >= l
        while (a < z) {
            const long long mid = (a + z) >> 1;
            if (cl(mid) >= l) z = mid;
            else a = mid + 1;
        }
        long long c = s, e = wr;  // last t with cl(t) >= l
        while (c < e) {
            const long long mid = (c + e + 1) >> 1;
            if (cl(mid) >= l) c = mid;
            else e = mid - 1;
        }
        const long long cc = c - a + 1;
        if (cc <= ncell) {
            const long long nch = (cc + leaf - 1) / leaf, off = s - a;
            return (off == 0) || ((off * nch) / cc != ((off - 1) * nch) / cc);
        }
    }
    // more than ncell identical keys: chunk the run of equal keys
    const unsigned long long *G = b.keys[0];
    long long a = lo, z = s;
    while (a < z) {
        long long mid = (a + z) >> 1;
        if (G[mid] < ks) a = mid + 1;
        else z = mid;
    }
    return ((s - a) % leaf) == 0;
}

// exclusive scan over the block (blockDim == kLeafThreads); total returned in *tot
__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();  // wsum free
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < kLeafThreads / 32; ++k) {
        const int t = wsum[k];
        if (k < w) before += t;
        all += t;
    }
    *tot = all;
    return before + x - v;
}

// Leaf counts of every problem and the layout of every tree level, by one
// block (exclusive scans over the problems, in chunks of the block size).
__device__ void problem_meta(const BatchView &b)
{
    __shared__ int run[kMaxLevels + 1];
    __shared__ int wsum[kLeafThreads / 32];
    if (threadIdx.x <= kMaxLevels) run[threadIdx.x] = 0;
    __syncthreads();
    for (int p0 = 0; p0 < b.nprob; p0 += blockDim.x) {
        const int p = p0 + threadIdx.x;
        int cnt[kMaxLevels + 1];
        for (int l = 0; l <= kMaxLevels; ++l) cnt[l] = 0;
        if (p < b.nprob) {
            const ProbStatic &ps = b.prob[p];
            if (ps.n > 0) {
                const int lb = (int)__ldcg(&b.flag[ps.base]) - 1;
                cnt[0] = (int)__ldcg(&b.flag[ps.base + ps.n - 1]) - lb;
            }
            for (int l = 1; l <= kMaxLevels; ++l)
                cnt[l] = cnt[l - 1] > kBranch ? (cnt[l - 1] + kBranch - 1) / kBranch : 0;
        }
        int top = 0;
        for (int l = 0; l <= kMaxLevels; ++l) {
            int tot;
            const int ex = block_excl_scan(cnt[l], wsum, &tot);
            if (p < b.nprob) {
                ProbDyn &d = b.dyn[p];
                d.node_off[l] = run[l] + ex;
                d.node_cnt[l] = cnt[l];
                if (l == 0) {
                    d.leaf_base = run[0] + ex;
                    d.nleaf = cnt[0];
                }
                if (cnt[l] > 0) top = l;
            }
            __syncthreads();
            if (threadIdx.x == 0) run[l] += tot;
        }
        if (p < b.nprob) b.dyn[p].top_level = top;
    }
    __syncthreads();
    if (threadIdx.x <= kMaxLevels) b.counters[1 + threadIdx.x] = run[threadIdx.x];
}

// Leaf start flags, their inclusive scan (the leaf index of every particle)
// with a decoupled look-back between tiles, the leaf starts and owners; the
// last block to finish lays out the leaves and tree levels of every problem
// and clears the tile state for the next build.
__global__ void __launch_bounds__(kLeafThreads) k_leaf_scan(BatchView b)
{
    __shared__ unsigned long long sk[kLeafTile + 2 * kHalo];
    __shared__ int wsum[kLeafThreads / 32];
    __shared__ unsigned s_tile, s_prefix;
    __shared__ int s_last;
    unsigned *ts = b.tile_state;  // [0] tile ticket, [1] finished tiles, [2 + t] status of tile t
    if (threadIdx.x == 0) s_tile = atomicAdd(&ts[0], 1u);
    __syncthreads();
    const unsigned tile = s_tile;
    const long long n = b.ntot;
    const long long base = (long long)tile * kLeafTile;
    const long long k0 = base - kHalo;
    for (int k = threadIdx.x; k < kLeafTile + 2 * kHalo; k += blockDim.x) {
        const long long g = k0 + k;
        sk[k] = (g >= 0 && g < n) ? b.keys[0][g] : 0ull;
    }
    __syncthreads();
    unsigned f[kLeafItems];
    int tsum = 0;
    const long long s0 = base + (long long)threadIdx.x * kLeafItems;
    for (int r = 0; r < kLeafItems; ++r) {
        f[r] = s0 + r < n ? leaf_flag(b, sk, k0, s0 + r) : 0u;
        tsum += (int)f[r];
    }
    int agg;
    const int ex = block_excl_scan(tsum, wsum, &agg);
    // decoupled look-back, 32 predecessors per round (warp 0)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        volatile unsigned *vs = ts + 2;
        unsigned prefix = 0;
        if (tile == 0) {
            if (lane == 0) {
                __threadfence();
                vs[0] = kTilePre | (unsigned)agg;
            }
        } else {
            if (lane == 0) vs[tile] = kTileAgg | (unsigned)agg;
            __threadfence();
            long long t = (long long)tile - 1, spins = 0;
            for (;;) {
                const long long tt = t - lane;
                const unsigned v = tt >= 0 ? (unsigned)vs[tt] : (unsigned)kTilePre;  // before tile 0: an empty prefix
                const unsigned pre = __ballot_sync(0xffffffffu, (v & kTilePre) != 0u);
                const unsigned pend = __ballot_sync(0xffffffffu, (v & ~kTileMask) == 0u);
                const int np = pre ? __ffs(pre) - 1 : 31;  // nearest inclusive prefix (or the window)
                const unsigned need = np == 31 ? 0xffffffffu : ((1u << (np + 1)) - 1u);
                if (pend & need) {
                    if (++spins > kTileSpinLimit) {
                        if (lane == 0) atomicExch(&b.counters[kTimeoutCounter], 1);  // reported as a timeout
                        break;
                    }
                    continue;
                }
                prefix += warp_sum(lane <= np ? (v & kTileMask) : 0u);
                if (pre) break;
                t -= 32;
            }
            if (lane == 0) {
                __threadfence();
                vs[tile] = kTilePre | (prefix + (unsigned)agg);
            }
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    unsigned run = s_prefix + (unsigned)ex;
    for (int r = 0; r < kLeafItems; ++r) {
        const long long s = s0 + r;
        if (s >= n) break;
        run += f[r];
        b.flag[s] = run;
        if (f[r]) {
            b.leaf_start[run - 1] = (int)s;
            b.leaf_pid[run - 1] = (int)(sk[s - k0] >> kMortonTotal);
        }
        if (s == n - 1) {
            b.leaf_start[run] = (int)n;
            b.counters[0] = (int)run;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ts[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) ts[2 + k] = 0u;
    if (threadIdx.x == 0) {
        ts[0] = 0u;
        ts[1] = 0u;
    }
    problem_meta(b);
}



template <typename T4, bool WRAP>
__global__ void k_leaf_props(BatchView b)
{
    const int nleaf = b.counters[0];
    if (blockIdx.x == 0)
        for (int p = threadIdx.x; p < b.nprob; p += blockDim.x) b.dyn[p].lists_stale = 0;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) leaf_props_one<T4, WRAP>(b, leaf);
}

// Smoothing-sphere boxes and h_max of the leaves after the density solve,
// in FP32 from the staged offsets and the float h (rounded up) the density
// solve left, widened for the offsets' rounding, plus the reference point
// rounded down (up) that the leaf pass kept.
template <typename T4>
__global__ void k_leaf_refit(BatchView b)
{
    // a block-step tick with tasks: unless some particle's final h outgrew
    // the prediction the leaf pass boxed it with (lists_stale), those boxes
    // already hold every smoothing sphere (the kept particles' h unchanged)
    if (b.block_on && b.block_tasks && !*(volatile int *)&b.dyn[0].lists_stale) return;
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        const int st = b.leaf_start[leaf], cnt = b.leaf_start[leaf + 1] - st;
        const bool on = lane < cnt;
        const PhysParams &ph = b.prob[b.leaf_pid[leaf]].ph;
        const float kr = ph.kr_f;
        float slo[3], shi[3], hm = 0.f, ex[3] = {0.f, 0.f, 0.f};
        if (on) {
            const T4 v = ((const T4 *)b.pm)[st + lane];
            const float o[3] = {offset_f(v.x), offset_f(v.y), offset_f(v.z)};
            const float h = b.hf[st + lane], h2 = __fmul_ru(kr, h);
            hm = h;
            for (int a = 0; a < 3; ++a) ex[a] = fabsf(o[a]);
            for (int a = 0; a < 3; ++a) {
                const float mag = __fadd_ru(fabsf(o[a]), h2);
                slo[a] = widen_dn(__fsub_rd(o[a], h2), mag);
                shi[a] = widen_up(__fadd_ru(o[a], h2), mag);
            }
        } else {
            for (int a = 0; a < 3; ++a) {
                slo[a] = INFINITY;
                shi[a] = -INFINITY;
            }
        }
        hm = warp_max(hm);
        const float ext = leaf_ext_bits(ex, ph);
        for (int a = 0; a < 3; ++a) {
            slo[a] = warp_min(slo[a]);
            shi[a] = warp_max(shi[a]);
        }
        float bl = 0.f, bh = 0.f;
        if (lane < 3) {
            bl = __fadd_rd(b.leaf_cf[6 * (long long)leaf + lane], axis_of(slo, lane));
            bh = __fadd_ru(b.leaf_cf[6 * (long long)leaf + 3 + lane], axis_of(shi, lane));
        }
        const float l0 = __shfl_sync(0xffffffffu, bl, 0), l1 = __shfl_sync(0xffffffffu, bl, 1),
                    l2 = __shfl_sync(0xffffffffu, bl, 2);
        const float h0 = __shfl_sync(0xffffffffu, bh, 0), h1 = __shfl_sync(0xffffffffu, bh, 1),
                    h2 = __shfl_sync(0xffffffffu, bh, 2);
        if (lane == 0) {
            NodeBox &nb = b.nodes[0][leaf];
            nb.plo.w = hm;
            nb.slo = make_float4(l0, l1, l2, ext);
            nb.shi = make_float4(h0, h1, h2, 0.f);
        }
        tree_up(b, leaf);
    }
}

int persistent_blocks(int threads)
{
    static int sms = 0;
    if (!sms) sms = dev_info().sm_count;
    return sms * (2048 / threads);
}

}  // namespace

long long leaves_upper_bound(long long n) { return n > 0 ? n : 1; }

int levels_needed(long long max_leaves)
{
    int l = 0;
    long long c = max_leaves;
    while (c > kBranch && l < kMaxLevels) {
        c = (c + kBranch - 1) / kBranch;
        ++l;
    }
    return l;
}

cudaError_t launch_gather(const BatchView &b, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    k_gather<<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_build_leaves(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    const long long tiles = (b.ntot + kLeafTile - 1) / kLeafTile;
    k_leaf_scan<<<(unsigned)tiles, kLeafThreads, 0, st>>>(b);
    int pb = persistent_blocks(256);
    if (precision == SPH_PREC_FP64) k_leaf_props<dbl4, false><<<pb, 256, 0, st>>>(b);
    else k_leaf_props<float4, false><<<pb, 256, 0, st>>>(b);
    return cudaGetLastError();
}

// Tree reuse (Sec. 4.2): the leaves of the last build keep their particles;
// offsets, leaf boxes and node boxes are recomputed from the new positions.
// Offsets are taken by minimum image, as a kept leaf may straddle a periodic
// boundary after particles moved.
cudaError_t launch_update_leaves(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    int pb = persistent_blocks(256);
    if (precision == SPH_PREC_FP64) k_leaf_props<dbl4, true><<<pb, 256, 0, st>>>(b);
    else k_leaf_props<float4, true><<<pb, 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_refit(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    int pb = persistent_blocks(256);
    if (precision == SPH_PREC_FP64) k_leaf_refit<dbl4><<<pb, 256, 0, st>>>(b);
    else k_leaf_refit<float4><<<pb, 256, 0, st>>>(b);
    return cudaGetLastError();
}

long long leaf_tiles(long long n) { return (n + kLeafTile - 1) / kLeafTile; }

}  // namespace sph
