// Leaf cells and the tree over them (Sec. 2.6, tree; Sec. 2.6 also the
// per-leaf neighbour walk).  The paper's KD tree with N_LEAF-particle leaves
// and per-cell "smallest box containing all the smoothing spheres" is
// replaced by:
//   - leaves = octree cells of the Morton order: for each particle the
//     coarsest cell holding at most 2*leaf_size particles of its problem,
//     split into ceil(count/leaf_size) equal consecutive chunks;
//   - an implicit 32-ary tree over each problem's leaves (32 consecutive
//     leaves per level-1 node, 32 level-1 nodes per level-2 node, ...), whose
//     nodes keep a position box and a smoothing-sphere box, both FP32 rounded
//     outwards from FP64 data.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

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
    b.sm[s] = ps.m[i];
    b.sh[s] = ps.h[i];
}

__device__ __forceinline__ int common_levels(unsigned long long a, unsigned long long b)
{
    unsigned x = (unsigned)((a ^ b) & ((1ull << kMortonTotal) - 1ull));
    if (x == 0u) return kMortonBits;
    return (__clz(x) - (32 - kMortonTotal)) / 3;
}

// Leaf start flags (see the file comment for the rule).
__global__ void k_leaf_flags(BatchView b)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.ntot) return;
    const unsigned long long *K = b.keys[0];
    const unsigned long long ks = K[s];
    const int p = (int)(ks >> kMortonTotal);
    const long long lo = b.prob[p].base, hi = lo + b.prob[p].n - 1;
    const int leaf = 32 / b.prob[p].lpp, ncell = 2 * leaf;
    long long pl = s - lo < ncell ? s - lo : ncell;
    long long pr = hi - s < ncell ? hi - s : ncell;
    int found = -1;
    for (int l = 0; l <= kMortonBits; ++l) {
        while (pl > 0 && common_levels(ks, K[s - pl]) < l) --pl;
        while (pr > 0 && common_levels(ks, K[s + pr]) < l) --pr;
        if (1 + pl + pr <= ncell) {
            found = l;
            break;
        }
    }
    unsigned flag;
    if (found >= 0) {
        long long cs = s - pl, cc = 1 + pl + pr;
        long long nch = (cc + leaf - 1) / leaf;
        long long off = s - cs;
        flag = (off == 0) || ((off * nch) / cc != ((off - 1) * nch) / cc);
    } else {
        // more than 2*leaf_size identical keys: chunk the run of equal keys
        long long a = lo, z = s;
        while (a < z) {
            long long mid = (a + z) >> 1;
            if (K[mid] < ks) a = mid + 1;
            else z = mid;
        }
        flag = ((s - a) % leaf) == 0;
    }
    b.flag[s] = flag;
}

// ---- inclusive scan of the flags (block sums, one-block scan, apply) ------
__global__ void k_scan_tile_sums(const unsigned *a, long long n, unsigned *sums)
{
    __shared__ unsigned red[kScanThreads / 32];
    long long base = (long long)blockIdx.x * kScanTile;
    unsigned s = 0;
    for (int r = 0; r < kScanItems; ++r) {
        long long k = base + r * kScanThreads + threadIdx.x;
        if (k < n) s += a[k];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_single_excl(unsigned *a, long long len)
{
    __shared__ unsigned part[1024];
    long long per = (len + blockDim.x - 1) / blockDim.x;
    long long lo = threadIdx.x * per, hi = lo + per < len ? lo + per : len;
    unsigned s = 0;
    for (long long k = lo; k < hi; ++k) s += a[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    unsigned run = part[threadIdx.x] - s;
    for (long long k = lo; k < hi; ++k) {
        unsigned v = a[k];
        a[k] = run;
        run += v;
    }
}

// Tile-local inclusive scan plus the tile offset; items are contiguous per
// thread (thread t owns items [t*8, t*8+8) of the tile).
__global__ void k_scan_apply(unsigned *a, long long n, const unsigned *offs)
{
    __shared__ unsigned part[kScanThreads];
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
    for (int r = 0; r < kScanItems; ++r) {
        long long k = base + r;
        v[r] = k < n ? a[k] : 0u;
        s += v[r];
        v[r] = s;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        unsigned t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    unsigned pre = offs[blockIdx.x] + part[threadIdx.x] - s;
    for (int r = 0; r < kScanItems; ++r) {
        long long k = base + r;
        if (k < n) a[k] = pre + v[r];
    }
}

__global__ void k_leaf_starts(BatchView b)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.ntot) return;
    unsigned inc = b.flag[s];
    bool start = (s == 0) || (b.flag[s - 1] != inc);
    if (start) {
        int leaf = (int)inc - 1;
        b.leaf_start[leaf] = (int)s;
        b.leaf_pid[leaf] = (int)(b.keys[0][s] >> kMortonTotal);
    }
    if (s == b.ntot - 1) {
        b.leaf_start[inc] = (int)b.ntot;
        b.counters[0] = (int)inc;
    }
}

// Leaf counts per problem and the layout of every tree level (one thread;
// the prefix over problems is serial and tiny).
__global__ void k_problem_meta(BatchView b)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int off[kMaxLevels + 1];
    for (int l = 0; l <= kMaxLevels; ++l) off[l] = 0;
    for (int p = 0; p < b.nprob; ++p) {
        ProbDyn &d = b.dyn[p];
        const ProbStatic &ps = b.prob[p];
        int nl = 0, lb = off[0];
        if (ps.n > 0) {
            lb = (int)b.flag[ps.base] - 1;
            nl = (int)b.flag[ps.base + ps.n - 1] - lb;
        }
        d.leaf_base = lb;
        d.nleaf = nl;
        d.node_cnt[0] = nl;
        d.node_off[0] = lb;
        off[0] = lb + nl;
        int top = 0;
        for (int l = 1; l <= kMaxLevels; ++l) {
            int c = d.node_cnt[l - 1] > kBranch ? (d.node_cnt[l - 1] + kBranch - 1) / kBranch : 0;
            d.node_cnt[l] = c;
            d.node_off[l] = off[l];
            off[l] += c;
            if (c > 0) top = l;
        }
        d.top_level = top;
    }
    for (int l = 0; l <= kMaxLevels; ++l) b.counters[1 + l] = off[l];
}

__device__ __forceinline__ float f_rd(double v) { return __double2float_rd(v); }
__device__ __forceinline__ float f_ru(double v) { return __double2float_ru(v); }

// Leaf reference point, position box and the offsets of its particles from
// that point.  The reference point is the leaf's first particle (FP64); the
// FP64 difference is taken before the cast to the staging precision, and the
// box is formed from the offsets (FP64 adds, rounded outwards to float).
template <typename T4>
__global__ void k_leaf_props(BatchView b)
{
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        int st = b.leaf_start[leaf], cnt = b.leaf_start[leaf + 1] - st;
        bool on = lane < cnt;
        double c[3] = {b.sx[st], b.sy[st], b.sz[st]};
        float o[3] = {0.f, 0.f, 0.f};
        double od[3] = {0.0, 0.0, 0.0};
        if (on) {
            od[0] = b.sx[st + lane] - c[0];
            od[1] = b.sy[st + lane] - c[1];
            od[2] = b.sz[st + lane] - c[2];
            for (int a = 0; a < 3; ++a) o[a] = (float)od[a];
            T4 v;
            v.x = (decltype(v.x))od[0];
            v.y = (decltype(v.y))od[1];
            v.z = (decltype(v.z))od[2];
            v.w = (decltype(v.w))b.sm[st + lane];
            ((T4 *)b.pm)[st + lane] = v;
        }
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(on ? o[a] : INFINITY);
            hi[a] = warp_max(on ? o[a] : -INFINITY);
        }
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) b.leaf_c[3 * (long long)leaf + a] = c[a];
            // float offsets are within one rounding of the FP64 ones: widen by it
            NodeBox nb;
            float l3[3], h3[3];
            for (int a = 0; a < 3; ++a) {
                double e = 1e-6 * ((double)fabsf(lo[a]) + (double)fabsf(hi[a])) + 1e-30;
                l3[a] = f_rd(c[a] + (double)lo[a] - e);
                h3[a] = f_ru(c[a] + (double)hi[a] + e);
            }
            nb.plo = make_float4(l3[0], l3[1], l3[2], 0.f);
            nb.phi = make_float4(h3[0], h3[1], h3[2], (float)cnt);
            nb.slo = nb.plo;
            nb.shi = nb.phi;
            b.nodes[0][leaf] = nb;
        }
    }
}

// Smoothing-sphere boxes and h_max of the leaves after the density solve,
// formed from the FP64 offsets to the leaf reference point (FP32 arithmetic
// on offsets, one FP64 add per axis, rounded outwards).
__global__ void k_leaf_refit(BatchView b)
{
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        int st = b.leaf_start[leaf], cnt = b.leaf_start[leaf + 1] - st;
        bool on = lane < cnt;
        double c[3] = {b.leaf_c[3 * (long long)leaf], b.leaf_c[3 * (long long)leaf + 1],
                       b.leaf_c[3 * (long long)leaf + 2]};
        float o[3] = {0.f, 0.f, 0.f}, h2 = 0.f;
        double h = 0.0;
        if (on) {
            o[0] = (float)(b.sx[st + lane] - c[0]);
            o[1] = (float)(b.sy[st + lane] - c[1]);
            o[2] = (float)(b.sz[st + lane] - c[2]);
            h = b.sh[st + lane];
            h2 = __double2float_ru(2.0 * h);
        }
        float hmax = warp_max(on ? __double2float_ru(h) : 0.f);
        float slo[3], shi[3];
        for (int a = 0; a < 3; ++a) {
            slo[a] = warp_min(on ? __fsub_rd(o[a], h2) : INFINITY);
            shi[a] = warp_max(on ? __fadd_ru(o[a], h2) : -INFINITY);
        }
        if (lane == 0) {
            NodeBox &nb = b.nodes[0][leaf];
            float l3[3], h3[3];
            for (int a = 0; a < 3; ++a) {
                double e = 1e-6 * ((double)fabsf(slo[a]) + (double)fabsf(shi[a])) + 1e-30;
                l3[a] = f_rd(c[a] + (double)slo[a] - e);
                h3[a] = f_ru(c[a] + (double)shi[a] + e);
            }
            nb.plo.w = hmax;
            nb.slo = make_float4(l3[0], l3[1], l3[2], 0.f);
            nb.shi = make_float4(h3[0], h3[1], h3[2], 0.f);
        }
    }
}

// One tree level: node box = union of its (up to 32) children's boxes.
__global__ void k_tree_level(BatchView b, int level)
{
    const int lane = threadIdx.x & 31;
    const int total = b.counters[1 + level];
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int G = w; G < total; G += nw) {
        // owning problem: last p with node_off[level] <= G and a non-empty level
        int lo = 0, hi = b.nprob - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (b.dyn[mid].node_off[level] <= G) lo = mid;
            else hi = mid - 1;
        }
        const ProbDyn &d = b.dyn[lo];
        int k = G - d.node_off[level];
        int ch = kBranch * k + lane;
        bool on = ch < d.node_cnt[level - 1];
        NodeBox c;
        if (on) c = b.nodes[level - 1][d.node_off[level - 1] + ch];
        float v[12];
        v[0] = on ? c.plo.x : INFINITY;
        v[1] = on ? c.plo.y : INFINITY;
        v[2] = on ? c.plo.z : INFINITY;
        v[3] = on ? c.phi.x : -INFINITY;
        v[4] = on ? c.phi.y : -INFINITY;
        v[5] = on ? c.phi.z : -INFINITY;
        v[6] = on ? c.slo.x : INFINITY;
        v[7] = on ? c.slo.y : INFINITY;
        v[8] = on ? c.slo.z : INFINITY;
        v[9] = on ? c.shi.x : -INFINITY;
        v[10] = on ? c.shi.y : -INFINITY;
        v[11] = on ? c.shi.z : -INFINITY;
        float hm = warp_max(on ? c.plo.w : 0.f);
        float cnt = warp_sum(on ? c.phi.w : 0.f);
        for (int a = 0; a < 3; ++a) {
            v[a] = warp_min(v[a]);
            v[3 + a] = warp_max(v[3 + a]);
            v[6 + a] = warp_min(v[6 + a]);
            v[9 + a] = warp_max(v[9 + a]);
        }
        if (lane == 0) {
            NodeBox nb;
            nb.plo = make_float4(v[0], v[1], v[2], hm);
            nb.phi = make_float4(v[3], v[4], v[5], cnt);
            nb.slo = make_float4(v[6], v[7], v[8], 0.f);
            nb.shi = make_float4(v[9], v[10], v[11], 0.f);
            b.nodes[level][G] = nb;
        }
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

static cudaError_t launch_tree_levels(const BatchView &b, cudaStream_t st)
{
    int L = levels_needed(b.max_leaves);
    for (int l = 1; l <= L; ++l) {
        long long cap = b.node_cap[l];
        long long warps = cap < 152LL * 32 ? cap : 152LL * 32;
        if (warps < 1) warps = 1;
        k_tree_level<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(b, l);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_leaves(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    const long long n = b.ntot;
    unsigned g256 = (unsigned)((n + 255) / 256);
    k_leaf_flags<<<g256, 256, 0, st>>>(b);
    int nt = (int)((n + kScanTile - 1) / kScanTile);
    k_scan_tile_sums<<<nt, kScanThreads, 0, st>>>(b.flag, n, b.scan_aux);
    k_scan_single_excl<<<1, 1024, 0, st>>>(b.scan_aux, nt);
    k_scan_apply<<<nt, kScanThreads, 0, st>>>(b.flag, n, b.scan_aux);
    k_leaf_starts<<<g256, 256, 0, st>>>(b);
    k_problem_meta<<<1, 32, 0, st>>>(b);
    int pb = persistent_blocks(256);
    if (precision == SPH_PREC_FP64) k_leaf_props<dbl4><<<pb, 256, 0, st>>>(b);
    else k_leaf_props<float4><<<pb, 256, 0, st>>>(b);
    return launch_tree_levels(b, st);
}

cudaError_t launch_refit(const BatchView &b, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    int pb = persistent_blocks(256);
    k_leaf_refit<<<pb, 256, 0, st>>>(b);
    return launch_tree_levels(b, st);
}

}  // namespace sph
