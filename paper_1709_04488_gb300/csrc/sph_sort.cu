// Morton keys and a stable LSD radix sort of (key, index) pairs.
//
// The paper builds a KD tree by recursive median bisection (Sec. 2.6, tree;
// Sec. 3.2 notes the serial top levels limit its parallel scaling).  Here the
// spatial order comes from one fully parallel sort instead: a 30-bit Morton
// key (10 bits per axis) per particle, prefixed by the problem index in a
// batch, sorted stably so that ties keep the original particle order.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per block
constexpr int kBboxThreads = 1024;

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
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

// Bounding box of isolated problems (FP64, ordered-integer atomics after a
// block reduction when the whole block belongs to one problem).
__global__ void k_bbox(BatchView b)
{
    __shared__ unsigned long long red[6][kBboxThreads / 32];
    __shared__ int uniform_p;
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int p = -1;
    unsigned long long v[6];
    for (int a = 0; a < 3; ++a) {
        v[a] = ~0ull;
        v[3 + a] = 0ull;
    }
    if (g < b.ntot) {
        p = find_problem(b.prob_base, b.nprob, g);
        const ProbStatic &ps = b.prob[p];
        if (!ps.ph.periodic) {
            long long i = g - ps.base;
            double X[3] = {ps.x[i], ps.y[i], ps.z[i]};
            for (int a = 0; a < 3; ++a) {
                v[a] = ordered_bits(X[a]);
                v[3 + a] = v[a];
            }
        } else {
            p = -2;  // nothing to do
        }
    }
    if (threadIdx.x == 0) uniform_p = p;
    __syncthreads();
    int p0 = uniform_p;
    bool uni = __syncthreads_and(p == p0 || p == -1);
    if (uni) {
        if (p0 < 0) return;
        for (int a = 0; a < 6; ++a) {
            unsigned long long x = v[a];
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                x = a < 3 ? (y < x ? y : x) : (y > x ? y : x);
            }
            if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = x;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            int nw = blockDim.x >> 5;
            for (int a = 0; a < 6; ++a) {
                unsigned long long x = threadIdx.x < nw ? red[a][threadIdx.x] : (a < 3 ? ~0ull : 0ull);
                for (int o = 16; o > 0; o >>= 1) {
                    unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                    x = a < 3 ? (y < x ? y : x) : (y > x ? y : x);
                }
                if (threadIdx.x == 0) {
                    if (a < 3) atomicMin(&b.dyn[p0].bbox_bits[a], x);
                    else atomicMax(&b.dyn[p0].bbox_bits[a], x);
                }
            }
        }
    } else if (p >= 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&b.dyn[p].bbox_bits[a], v[a]);
            atomicMax(&b.dyn[p].bbox_bits[3 + a], v[3 + a]);
        }
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

__global__ void k_keys(BatchView b)
{
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.ntot) return;
    int p = find_problem(b.prob_base, b.nprob, g);
    const ProbStatic &ps = b.prob[p];
    const ProbDyn &d = b.dyn[p];
    long long i = g - ps.base;
    double X[3] = {ps.x[i], ps.y[i], ps.z[i]};
    unsigned code = 0;
    for (int a = 0; a < 3; ++a) {
        double t = (X[a] - d.dom_lo[a]) * d.dom_inv * (double)(1 << kMortonBits);
        int c = t > 0.0 ? (int)t : 0;  // NaN maps to 0
        c = c > (1 << kMortonBits) - 1 ? (1 << kMortonBits) - 1 : c;
        code |= spread10((unsigned)c) << a;
    }
    b.keys[0][g] = ((unsigned long long)p << kMortonTotal) | code;
    b.vals[0][g] = (unsigned)g;
}

// ---- radix sort: per-tile digit histograms, one scan, stable scatter -----
__global__ void k_radix_hist(const unsigned long long *keys, long long n, int shift, unsigned *hist,
                             int nblk)
{
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        long long k = base + r * kSortThreads + threadIdx.x;
        if (k < n) atomicAdd(&cnt[(unsigned)(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of `len` values in place with one block of 1024 threads.
__global__ void k_scan_single(unsigned *a, long long len)
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

// Stable scatter: items of a tile are ranked in index order (round-major,
// thread-minor), warp peers found with __match_any_sync, warps combined
// through shared per-warp digit counts.
__global__ void k_radix_scatter(const unsigned long long *kin, const unsigned *vin,
                                unsigned long long *kout, unsigned *vout, long long n, int shift,
                                const unsigned *hist, int nblk, int identity_vals)
{
    constexpr int NW = kSortThreads / 32;
    __shared__ unsigned run[256];
    __shared__ unsigned wcnt[NW][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = hist[(long long)threadIdx.x * nblk + blockIdx.x];
    for (int w = 0; w < NW; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        long long k = base + r * kSortThreads + threadIdx.x;
        bool ok = k < n;
        unsigned long long key = ok ? kin[k] : 0ull;
        unsigned val = ok ? (identity_vals ? (unsigned)k : vin[k]) : 0u;
        unsigned d = ok ? (unsigned)(key >> shift) & 255u : 256u + lane;  // unique dummies
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
            tot += wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = 0;
        }
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

__global__ void k_copy_perm(const unsigned *vals, int *perm, long long n)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) perm[k] = (int)vals[k];
}

}  // namespace

cudaError_t launch_domain_and_keys(const BatchView &b, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    int pb = (b.nprob + 127) / 128;
    k_reset_bbox<<<pb, 128, 0, st>>>(b.dyn, b.nprob);
    long long nb = (b.ntot + kBboxThreads - 1) / kBboxThreads;
    k_bbox<<<(unsigned)nb, kBboxThreads, 0, st>>>(b);
    k_domain<<<pb, 128, 0, st>>>(b);
    k_keys<<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_radix_sort(const BatchView &b, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    const long long n = b.ntot;
    const int nblk = (int)((n + kSortTile - 1) / kSortTile);
    const int passes = (b.key_bits + 7) / 8;
    int src = 0;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = 8 * pass;
        k_radix_hist<<<nblk, kSortThreads, 0, st>>>(b.keys[src], n, shift, b.hist, nblk);
        k_scan_single<<<1, 1024, 0, st>>>(b.hist, 256LL * nblk);
        k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(b.keys[src], b.vals[src], b.keys[src ^ 1],
                                                       b.vals[src ^ 1], n, shift, b.hist, nblk, 0);
        src ^= 1;
    }
    k_copy_perm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b.vals[src], b.perm, n);
    if (src != 0) {
        // leave the sorted keys in keys[0] for the leaf builder
        cudaMemcpyAsync(b.keys[0], b.keys[1], sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

}  // namespace sph
