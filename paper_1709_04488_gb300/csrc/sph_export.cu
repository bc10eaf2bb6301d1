// Exact FP64 neighbour lists (CSR, ids ascending) for one problem: the
// per-leaf tree walk retrieves the candidates (Sec. 4.2), membership is
// decided on absolute FP64 positions with the periodic minimum image and
// r^2 = dx*dx + dy*dy + dz*dz formed without fused multiply-add, compared
// with (R_K h)^2 (gather list) or (R_K max(h_i,h_j))^2 (force list), R_K the
// kernel's support in units of h (2 for M4, 3 for M6).  Used by
// the tests to compare neighbour sets bit for bit with the CPU oracle.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kExportCap = 1024;  // neighbours one particle may have in the export

__device__ __forceinline__ bool axis_overlap_x(float alo, float ahi, float blo, float bhi, float R, int periodic,
                                               float L)
{
    float ca = 0.5f * (alo + ahi), ha = 0.5f * (ahi - alo);
    float cb = 0.5f * (blo + bhi), hb = 0.5f * (bhi - blo);
    float reach = ha + hb + R;
    reach += 2e-6f * (fabsf(ca) + fabsf(cb) + reach) + 1e-30f;
    float d = fabsf(ca - cb);
    if (periodic) {
        if (reach >= 0.5f * L) return true;
        if (d > L) d -= L;
        d = fminf(d, L - d);
    }
    return d <= reach;
}

__device__ __forceinline__ bool overlap_x(const float4 &alo, const float4 &ahi, const float4 &blo, const float4 &bhi,
                                          float R, const PhysParams &ph)
{
    return axis_overlap_x(alo.x, ahi.x, blo.x, bhi.x, R, ph.periodic, (float)ph.box_len[0]) &&
           axis_overlap_x(alo.y, ahi.y, blo.y, bhi.y, R, ph.periodic, (float)ph.box_len[1]) &&
           axis_overlap_x(alo.z, ahi.z, blo.z, bhi.z, R, ph.periodic, (float)ph.box_len[2]);
}

__global__ void k_set_sorted_h(BatchView b, const double *h_in)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.ntot) return;
    int p = (int)(b.keys[0][s] >> kMortonTotal);
    long long i = (long long)b.perm[s] - b.prob[p].base;
    const double h = h_in ? h_in[i] : b.prob[p].h[i];
    b.sh[s] = h;
    b.hf[s] = __double2float_ru(h);
}

// pass 0: count into cnt[i]; pass 1: write sorted ids at offsets[i]
__global__ void __launch_bounds__(128) k_export(BatchView b, int kind, int pass, unsigned *cnt,
                                                const long long *offsets, int *idx, long long cap)
{
    __shared__ int buf[4][kExportCap];
    __shared__ int sorted[4][kExportCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const ProbStatic &ps = b.prob[0];
    const ProbDyn &d = b.dyn[0];
    const PhysParams &ph = ps.ph;
    for (long long s = w; s < b.ntot; s += nw) {
        const double xi = b.sx[s], yi = b.sy[s], zi = b.sz[s], hi = b.sh[s];
        const long long i = (long long)b.perm[s] - ps.base;
        float4 qlo = make_float4(__double2float_rd(xi), __double2float_rd(yi), __double2float_rd(zi), 0.f);
        float4 qhi = make_float4(__double2float_ru(xi), __double2float_ru(yi), __double2float_ru(zi), 0.f);
        const float R = __double2float_ru(ph.kr * hi) * 1.0001f;
        int n = 0;
        // walk (same structure as the pair kernels)
        const int top = d.top_level;
        unsigned mask[kMaxLevels + 1];
        int base[kMaxLevels + 1];
        auto test = [&](const NodeBox &nb) {
            bool t = overlap_x(qlo, qhi, nb.plo, nb.phi, R, ph);
            if (kind == 1) t = t || overlap_x(qlo, qhi, nb.slo, nb.shi, 0.f, ph);
            return t;
        };
        int lvl = top;
        base[top] = 0;
        mask[top] = __ballot_sync(FULL, lane < d.node_cnt[top] && test(b.nodes[top][d.node_off[top] + lane]));
        for (;;) {
            unsigned m = mask[lvl];
            if (m == 0u) {
                if (++lvl > top) break;
                continue;
            }
            int c = __ffs(m) - 1;
            mask[lvl] = m & (m - 1u);
            int node = base[lvl] + c;
            if (lvl == 0) {
                int B = d.node_off[0] + node;
                int stB = b.leaf_start[B], nB = b.leaf_start[B + 1] - stB;
                bool hit = false;
                int jid = 0;
                if (lane < nB) {
                    long long j = stB + lane;
                    double dx = min_image(__dsub_rn(xi, b.sx[j]), ph.box_len[0], ph.periodic);
                    double dy = min_image(__dsub_rn(yi, b.sy[j]), ph.box_len[1], ph.periodic);
                    double dz = min_image(__dsub_rn(zi, b.sz[j]), ph.box_len[2], ph.periodic);
                    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    double hh = kind == 1 ? fmax(hi, b.sh[j]) : hi;
                    const double Rk = __dmul_rn(ph.kr, hh);  // R_K h, rounded as the oracle's
                    double R2 = __dmul_rn(Rk, Rk);
                    hit = r2 < R2 && !(kind == 1 && j == s);
                    jid = (int)((long long)b.perm[j] - ps.base);
                }
                unsigned hm = __ballot_sync(FULL, hit);
                if (pass == 1 && hit) {
                    int pos = n + __popc(hm & ((1u << lane) - 1u));
                    if (pos < kExportCap) buf[wib][pos] = jid;
                }
                n += __popc(hm);
                continue;
            }
            int ch = node * kBranch + lane;
            bool ok = ch < d.node_cnt[lvl - 1] && test(b.nodes[lvl - 1][d.node_off[lvl - 1] + ch]);
            --lvl;
            base[lvl] = node * kBranch;
            mask[lvl] = __ballot_sync(FULL, ok);
        }
        if (pass == 0) {
            if (lane == 0) cnt[i] = (unsigned)n;
            continue;
        }
        __syncwarp();
        int nn = n < kExportCap ? n : kExportCap;
        if (n > kExportCap && lane == 0) atomicOr(&ps.diag->status, ST_OVERFLOW);
        // rank sort (ids are distinct)
        for (int e = lane; e < nn; e += 32) {
            int v = buf[wib][e], r = 0;
            for (int f = 0; f < nn; ++f) r += buf[wib][f] < v;
            sorted[wib][r] = v;
        }
        __syncwarp();
        long long o = offsets[i];
        for (int e = lane; e < nn; e += 32)
            if (o + e < cap) idx[o + e] = sorted[wib][e];
        __syncwarp();
    }
}

// exclusive scan of n counts into int64 offsets (one block; test-sized inputs)
__global__ void k_offsets(const unsigned *cnt, long long n, long long *offsets, long long *total)
{
    __shared__ long long part[1024];
    long long per = (n + blockDim.x - 1) / blockDim.x;
    long long lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
    long long s = 0;
    for (long long k = lo; k < hi; ++k) s += cnt[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        long long t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - s;
    for (long long k = lo; k < hi; ++k) {
        offsets[k] = run;
        run += cnt[k];
    }
    if (threadIdx.x == blockDim.x - 1) {
        offsets[n] = part[threadIdx.x];
        *total = part[threadIdx.x];
    }
}

}  // namespace

cudaError_t launch_set_sorted_h(const BatchView &b, const double *h_in, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    k_set_sorted_h<<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b, h_in);
    return cudaGetLastError();
}

cudaError_t launch_neighbour_export(const BatchView &b, int kind, const double *h_in, long long *offsets,
                                    int *idx, long long cap, long long *total_dev, cudaStream_t st)
{
    (void)h_in;
    if (b.ntot == 0) {
        cudaMemsetAsync(offsets, 0, sizeof(long long), st);
        cudaMemsetAsync(total_dev, 0, sizeof(long long), st);
        return cudaGetLastError();
    }
    unsigned *cnt = b.flag;  // reuse: the leaf flags are no longer needed
    int grid = dev_info().sm_count * 4;
    k_export<<<grid, 128, 0, st>>>(b, kind, 0, cnt, offsets, idx, cap);
    k_offsets<<<1, 1024, 0, st>>>(cnt, b.ntot, offsets, total_dev);
    k_export<<<grid, 128, 0, st>>>(b, kind, 1, cnt, offsets, idx, cap);
    return cudaGetLastError();
}

}  // namespace sph
