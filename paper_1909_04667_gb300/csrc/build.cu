// Oct-tree construction on the GPU (paper Sec. 3.1).
//
// The paper inserts particles one at a time and splits every leaf that would
// hold two of them.  The cells that exist at the end do not depend on the
// insertion order -- a cell exists when its parent holds more than the leaf
// bucket B -- so the same tree is built here in parallel from sorted keys:
//
//   1. root cube and 21-bit integer cell coordinates -> 63-bit Morton keys
//   2. stable radix sort of (key, particle index)
//   3. level by level, every cell holding more than B particles is split into
//      its non-empty octants (binary search of the sorted keys), children in
//      ascending octant order
//   4. FP64 masses and mass-weighted positions summed bottom-up, children in
//      ascending octant order and a leaf's particles in sorted order, with
//      explicit round-to-nearest operations (no contraction), so the result
//      is the same bit for bit on any correct implementation of that order
//   5. depth-first pre-order tables for the walk: per node the FP32 geometric
//      centre (exact: it lies on the 2^-22 L0 grid), side, centre of mass
//      relative to the centre, mass, skip index, particle range and leaf flag
//      -- three 16-byte records loaded with one vector load each -- and per
//      sorted particle its position relative to its leaf centre plus mass.
#include <cub/cub.cuh>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// Order-preserving map of a double to a signed 64-bit integer (for atomic
// min / max of doubles).
__device__ __forceinline__ long long ordered_bits(double v) {
    long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__host__ __device__ inline double from_ordered_bits(long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b >= 0 ? b : (b ^ 0x7fffffffffffffffLL));
#else
    long long r = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
    double d;
    memcpy(&d, &r, sizeof d);
    return d;
#endif
}

// Copies positions and masses into the system, applies the periodic shift and
// wrap, checks finiteness and ranges, and reduces the bounding box.
__global__ void k_prepare(const double *__restrict__ pin, const float *__restrict__ mass_in, int64_t n, int periodic,
                          double box, double s0, double s1, double s2, double *__restrict__ pout,
                          float *__restrict__ mout, long long *__restrict__ bbox, int *__restrict__ bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    long long lo[3], hi[3];
    bool have = i < n;
    if (have) {
        const double sh[3] = {s0, s1, s2};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double v = pin[3 * i + a];
            if (!isfinite(v))
                atomicOr(bad, 1);
            if (periodic) {
                if (!(v >= 0.0 && v < box))
                    atomicOr(bad, 2);
                v = __dadd_rn(v, __dmul_rn(sh[a], box));
                if (v >= box)
                    v = __dsub_rn(v, box);
            }
            pout[3 * i + a] = v;
            lo[a] = hi[a] = ordered_bits(v);
        }
        float m = mass_in[i];
        if (!(m > 0.0f) || !isfinite(m))
            atomicOr(bad, 4);
        mout[i] = m;
    }
    // warp-level min / max, then one atomic per warp
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long l = have ? lo[a] : LLONG_MAX, h = have ? hi[a] : LLONG_MIN;
        for (int o = 16; o > 0; o >>= 1) {
            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bbox[a], l);
            atomicMax(&bbox[3 + a], h);
        }
    }
}

// Spreads the low 21 bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint32_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x001f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x001f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// K1: Morton keys of the 21-bit cell coordinates q = floor((x - x0) 2^21 / L0).
__global__ void k_keys(const double *__restrict__ pos, int64_t n, double x0, double y0, double z0, double scale,
                       uint64_t *__restrict__ key, uint32_t *__restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double o[3] = {x0, y0, z0};
    uint64_t k = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double f = floor(__dmul_rn(__dsub_rn(pos[3 * i + a], o[a]), scale));
        long long q = (long long)f;
        if (f < 0.0)
            q = 0;
        if (f > (double)((1 << kMaxLevel) - 1))
            q = (1 << kMaxLevel) - 1;
        k |= spread3((uint64_t)q) << a;
    }
    key[i] = k;
    idx[i] = (uint32_t)i;
}

__global__ void k_rank(const uint32_t *__restrict__ perm, int64_t n, uint32_t *__restrict__ rank) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n)
        rank[perm[s]] = (uint32_t)s;
}

// first index in [lo, hi) whose key is >= bound (keys ascending)
__device__ __forceinline__ uint32_t lower_bound_key(const uint64_t *__restrict__ key, uint32_t lo, uint32_t hi,
                                                    uint64_t bound) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (key[mid] < bound)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

struct LevelArrays {
    uint32_t *first, *count, *child, *nchild;
    uint8_t *level;
    uint64_t *prefix;
};

// K3a: number of non-empty octants of each cell of one level that is split.
__global__ void k_count_children(const uint64_t *__restrict__ key, LevelArrays b, int64_t ls, int64_t lc, int level,
                                 int bucket, uint32_t *__restrict__ nch) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= lc)
        return;
    int64_t node = ls + i;
    uint32_t f = b.first[node], c = b.count[node];
    if ((int)c <= bucket || level >= kMaxLevel) {
        nch[i] = 0;
        return;
    }
    int shift = 3 * (kMaxLevel - level - 1);
    uint64_t base = b.prefix[node] << 3;
    uint32_t lo = f, end = f + c, k = 0;
    for (int o = 0; o < 8; o++) {
        uint32_t hi = (o == 7) ? end : lower_bound_key(key, lo, end, (base | (uint64_t)(o + 1)) << shift);
        k += hi > lo;
        lo = hi;
    }
    nch[i] = k;
}

// K3b: writes the children of one level (ascending octant) and each cell's
// child range.
__global__ void k_emit_children(const uint64_t *__restrict__ key, LevelArrays b, int64_t ls, int64_t lc, int level,
                                int bucket, const uint32_t *__restrict__ offs, int64_t next_start) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= lc)
        return;
    int64_t node = ls + i;
    uint32_t f = b.first[node], c = b.count[node];
    if ((int)c <= bucket || level >= kMaxLevel) {
        b.child[node] = 0;
        b.nchild[node] = 0;
        return;
    }
    int shift = 3 * (kMaxLevel - level - 1);
    uint64_t base = b.prefix[node] << 3;
    int64_t out = next_start + offs[i];
    b.child[node] = (uint32_t)out;
    uint32_t lo = f, end = f + c, k = 0;
    for (int o = 0; o < 8; o++) {
        uint32_t hi = (o == 7) ? end : lower_bound_key(key, lo, end, (base | (uint64_t)(o + 1)) << shift);
        if (hi > lo) {
            int64_t ch = out + k;
            b.first[ch] = lo;
            b.count[ch] = hi - lo;
            b.level[ch] = (uint8_t)(level + 1);
            b.prefix[ch] = base | (uint64_t)o;
            k++;
        }
        lo = hi;
    }
    b.nchild[node] = k;
}

// K4: FP64 monopoles of one level, children first (ascending octant), a
// leaf's particles in sorted order; explicit round-to-nearest adds / muls.
__global__ void k_multipole(LevelArrays b, int64_t ls, int64_t lc, const uint32_t *__restrict__ perm,
                            const double *__restrict__ pos, const float *__restrict__ mass, double *__restrict__ M,
                            double *__restrict__ S) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= lc)
        return;
    int64_t node = ls + i;
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    uint32_t nc = b.nchild[node];
    if (nc == 0) {
        uint32_t f = b.first[node], e = f + b.count[node];
        for (uint32_t s = f; s < e; s++) {
            uint32_t j = perm[s];
            double mj = (double)mass[j];
            m = __dadd_rn(m, mj);
            sx = __dadd_rn(sx, __dmul_rn(mj, pos[3 * j]));
            sy = __dadd_rn(sy, __dmul_rn(mj, pos[3 * j + 1]));
            sz = __dadd_rn(sz, __dmul_rn(mj, pos[3 * j + 2]));
        }
    } else {
        uint32_t c0 = b.child[node];
        for (uint32_t c = c0; c < c0 + nc; c++) {
            m = __dadd_rn(m, M[c]);
            sx = __dadd_rn(sx, S[3 * c]);
            sy = __dadd_rn(sy, S[3 * c + 1]);
            sz = __dadd_rn(sz, S[3 * c + 2]);
        }
    }
    M[node] = m;
    S[3 * node] = sx;
    S[3 * node + 1] = sy;
    S[3 * node + 2] = sz;
}

__global__ void k_preorder_keys(LevelArrays b, int64_t total, uint64_t *__restrict__ okey, uint32_t *__restrict__ oval) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total)
        return;
    okey[i] = ((uint64_t)b.first[i] << 5) | (uint64_t)b.level[i];
    oval[i] = (uint32_t)i;
}

struct NodeOut {
    float4 *cen, *com;
    int4 *link;
    uint8_t *level;
    uint64_t *prefix;
    double *mass, *comd;
};

// K5: pre-order node tables.  skip(p) = number of nodes whose (first, level)
// key precedes (first + count, 0): the first node after p's subtree.
__global__ void k_finalize(LevelArrays b, const uint64_t *__restrict__ pkey, const uint32_t *__restrict__ pre2bfs,
                           int64_t total, const double *__restrict__ M, const double *__restrict__ S, double x0,
                           double y0, double z0, double L0, NodeOut o) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= total)
        return;
    uint32_t bi = pre2bfs[p];
    uint32_t f = b.first[bi], c = b.count[bi];
    int lvl = b.level[bi];
    uint64_t pre = b.prefix[bi];
    // skip: lower bound of (f + c) << 5 in the sorted pre-order keys after p
    uint64_t bound = (uint64_t)(f + c) << 5;
    int64_t lo = p + 1, hi = total;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (pkey[mid] < bound)
            lo = mid + 1;
        else
            hi = mid;
    }
    int leaf = b.nchild[bi] == 0;
    double m = M[bi];
    double cx = __ddiv_rn(S[3 * bi], m), cy = __ddiv_rn(S[3 * bi + 1], m), cz = __ddiv_rn(S[3 * bi + 2], m);
    uint32_t ix = compact3(pre), iy = compact3(pre >> 1), iz = compact3(pre >> 2);
    double half = ldexp(L0, -(lvl + 1));  // half side
    double rx = (double)(2 * (uint64_t)ix + 1) * half, ry = (double)(2 * (uint64_t)iy + 1) * half,
           rz = (double)(2 * (uint64_t)iz + 1) * half;  // centre relative to x0 (exact)
    o.cen[p] = make_float4((float)rx, (float)ry, (float)rz, (float)(2.0 * half));
    o.com[p] = make_float4((float)__dsub_rn(cx, __dadd_rn(x0, rx)), (float)__dsub_rn(cy, __dadd_rn(y0, ry)),
                           (float)__dsub_rn(cz, __dadd_rn(z0, rz)), (float)m);
    o.link[p] = make_int4((int)lo, (int)f, (int)c, leaf);
    o.level[p] = (uint8_t)lvl;
    o.prefix[p] = pre;
    o.mass[p] = m;
    o.comd[3 * p] = cx;
    o.comd[3 * p + 1] = cy;
    o.comd[3 * p + 2] = cz;
}

// Leaf particles relative to their leaf centre (FP64 difference -> FP32).
__global__ void k_leaf_particles(const float4 *__restrict__ cen, const int4 *__restrict__ link, int64_t total,
                                 const uint32_t *__restrict__ perm, const double *__restrict__ pos,
                                 const float *__restrict__ mass, double x0, double y0, double z0,
                                 float4 *__restrict__ spart) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= total)
        return;
    int4 l = link[p];
    if (!l.w)
        return;
    float4 c = cen[p];
    double ax = __dadd_rn(x0, (double)c.x), ay = __dadd_rn(y0, (double)c.y), az = __dadd_rn(z0, (double)c.z);
    for (int s = l.y; s < l.y + l.z; s++) {
        uint32_t j = perm[s];
        spart[s] = make_float4((float)__dsub_rn(pos[3 * j], ax), (float)__dsub_rn(pos[3 * j + 1], ay),
                               (float)__dsub_rn(pos[3 * j + 2], az), mass[j]);
    }
}

double pow2_ceil(double x) {
    int e;
    double f = std::frexp(x, &e);
    return (f == 0.5) ? std::ldexp(1.0, e - 1) : std::ldexp(1.0, e);
}

}  // namespace

int build_tree_device(Ctx *c, System *s, const double *pos_in, const float *mass_in, cudaStream_t st) {
    const int64_t n = s->n;
    const int B = s->bp.leaf_bucket;
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};

    TPM_CHECK(s->mem.get(&s->pos, 3 * n, st));
    TPM_CHECK(s->mem.get(&s->mass, n, st));
    TPM_CHECK(s->mem.get(&s->key, n, st));
    TPM_CHECK(s->mem.get(&s->perm, n, st));
    TPM_CHECK(s->mem.get(&s->rank, n, st));
    TPM_CHECK(s->mem.get(&s->spart, n, st));

    // ---- prepare, bounding box
    long long *bbox;
    int *bad;
    TPM_CHECK(tmp.get(&bbox, 6, st));
    TPM_CHECK(tmp.get(&bad, 1, st));
    long long init[6] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN};
    long long *h_bbox;
    TPM_CUDA(cudaMallocHost(&h_bbox, 8 * sizeof(long long)));
    struct HostGuard {
        void *p;
        ~HostGuard() { cudaFreeHost(p); }
    } hg{h_bbox};
    memcpy(h_bbox, init, sizeof init);
    TPM_CUDA(cudaMemcpyAsync(bbox, h_bbox, 6 * sizeof(long long), cudaMemcpyHostToDevice, st));
    TPM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_prepare<<<blocks_for(n), kThreads, 0, st>>>(pos_in, mass_in, n, s->bp.periodic, s->bp.box, s->bp.shift[0],
                                                   s->bp.shift[1], s->bp.shift[2], s->pos, s->mass, bbox, bad);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cudaMemcpyAsync(h_bbox, bbox, 6 * sizeof(long long), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaMemcpyAsync(h_bbox + 6, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaStreamSynchronize(st));
    int badv = (int)(h_bbox[6] & 0xffffffff);
    if (badv & 1) {
        set_error("non-finite position");
        return TPM_ENAN;
    }
    if (badv & 4) {
        set_error("masses must be finite and > 0");
        return TPM_ENAN;
    }
    if (badv & 2) {
        set_error("periodic positions must lie in [0, box)");
        return TPM_EINVAL;
    }

    // ---- root
    if (s->bp.periodic) {
        s->x0[0] = s->x0[1] = s->x0[2] = 0.0;
        s->L0 = s->bp.box;
    } else {
        double lo[3], hi[3], ext = 0.0;
        for (int a = 0; a < 3; a++) {
            lo[a] = from_ordered_bits(h_bbox[a]);
            hi[a] = from_ordered_bits(h_bbox[3 + a]);
            ext = std::max(ext, hi[a] - lo[a]);
        }
        if (!(ext > 0.0))
            ext = 1.0;
        double L0 = pow2_ceil(1.25 * ext);
        double unit = std::ldexp(L0, -kMaxLevel);
        for (int a = 0; a < 3; a++) {
            double slack = L0 - (hi[a] - lo[a]);
            double x0 = lo[a] - s->bp.shift[a] * slack;
            s->x0[a] = std::floor(x0 / unit) * unit;
        }
        s->L0 = L0;
    }

    // ---- keys and sort
    uint64_t *key_raw;
    uint32_t *idx_raw;
    TPM_CHECK(tmp.get(&key_raw, n, st));
    TPM_CHECK(tmp.get(&idx_raw, n, st));
    double scale = std::ldexp(1.0, kMaxLevel) / s->L0;
    k_keys<<<blocks_for(n), kThreads, 0, st>>>(s->pos, n, s->x0[0], s->x0[1], s->x0[2], scale, key_raw, idx_raw);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    size_t sort_bytes = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, key_raw, s->key, idx_raw, s->perm, (int)n, 0,
                                             3 * kMaxLevel, st));
    // the scan over one level reuses the same scratch
    size_t scan_bytes = 0;
    TPM_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (uint32_t *)nullptr, (uint32_t *)nullptr, (int)n, st));
    void *cub_tmp;
    size_t cub_bytes = std::max(sort_bytes, scan_bytes);
    TPM_CHECK(tmp.get((char **)&cub_tmp, cub_bytes, st));
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp, sort_bytes, key_raw, s->key, idx_raw, s->perm, (int)n, 0,
                                             3 * kMaxLevel, st));
    count_cub_call();
    k_rank<<<blocks_for(n), kThreads, 0, st>>>(s->perm, n, s->rank);
    count_launch();
    TPM_CUDA(cudaGetLastError());

    // ---- levels (breadth-first arrays)
    int64_t cap = 2 * n + 1024;
    LevelArrays b{};
    AllocSet bfs;
    bfs.ctx = c;
    struct BfsGuard {
        AllocSet &t;
        cudaStream_t st;
        ~BfsGuard() { t.release(st); }
    } bguard{bfs, st};
    auto alloc_bfs = [&](int64_t capacity, LevelArrays &out) -> int {
        TPM_CHECK(bfs.get(&out.first, capacity, st));
        TPM_CHECK(bfs.get(&out.count, capacity, st));
        TPM_CHECK(bfs.get(&out.child, capacity, st));
        TPM_CHECK(bfs.get(&out.nchild, capacity, st));
        TPM_CHECK(bfs.get(&out.level, capacity, st));
        TPM_CHECK(bfs.get(&out.prefix, capacity, st));
        return TPM_OK;
    };
    TPM_CHECK(alloc_bfs(cap, b));
    uint32_t *nch, *offs;
    TPM_CHECK(tmp.get(&nch, n + 1, st));
    TPM_CHECK(tmp.get(&offs, n + 1, st));
    {
        uint32_t zero = 0, cnt = (uint32_t)n;
        uint8_t l0 = 0;
        uint64_t p0 = 0;
        TPM_CUDA(cudaMemcpyAsync(b.first, &zero, 4, cudaMemcpyHostToDevice, st));
        TPM_CUDA(cudaMemcpyAsync(b.count, &cnt, 4, cudaMemcpyHostToDevice, st));
        TPM_CUDA(cudaMemcpyAsync(b.level, &l0, 1, cudaMemcpyHostToDevice, st));
        TPM_CUDA(cudaMemcpyAsync(b.prefix, &p0, 8, cudaMemcpyHostToDevice, st));
    }
    std::vector<int64_t> lstart{0}, lcount{1};
    uint32_t *h_tot = (uint32_t *)h_bbox;  // reuse pinned scratch
    for (int level = 0;; level++) {
        int64_t ls = lstart.back(), lc = lcount.back();
        k_count_children<<<blocks_for(lc), kThreads, 0, st>>>(s->key, b, ls, lc, level, B, nch);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        size_t sb = scan_bytes;
        TPM_CUDA(cub::DeviceScan::ExclusiveSum(cub_tmp, sb, nch, offs, (int)lc, st));
        count_cub_call();
        TPM_CUDA(cudaMemcpyAsync(h_tot, offs + lc - 1, 4, cudaMemcpyDeviceToHost, st));
        TPM_CUDA(cudaMemcpyAsync(h_tot + 1, nch + lc - 1, 4, cudaMemcpyDeviceToHost, st));
        TPM_CUDA(cudaStreamSynchronize(st));
        int64_t total = (int64_t)h_tot[0] + (int64_t)h_tot[1];
        int64_t next = ls + lc;
        if (next + total > cap) {
            int64_t ncap = std::max(next + total, cap + cap / 2);
            LevelArrays nb{};
            TPM_CHECK(alloc_bfs(ncap, nb));
            TPM_CUDA(cudaMemcpyAsync(nb.first, b.first, next * 4, cudaMemcpyDeviceToDevice, st));
            TPM_CUDA(cudaMemcpyAsync(nb.count, b.count, next * 4, cudaMemcpyDeviceToDevice, st));
            TPM_CUDA(cudaMemcpyAsync(nb.child, b.child, next * 4, cudaMemcpyDeviceToDevice, st));
            TPM_CUDA(cudaMemcpyAsync(nb.nchild, b.nchild, next * 4, cudaMemcpyDeviceToDevice, st));
            TPM_CUDA(cudaMemcpyAsync(nb.level, b.level, next, cudaMemcpyDeviceToDevice, st));
            TPM_CUDA(cudaMemcpyAsync(nb.prefix, b.prefix, next * 8, cudaMemcpyDeviceToDevice, st));
            b = nb;
            cap = ncap;
        }
        k_emit_children<<<blocks_for(lc), kThreads, 0, st>>>(s->key, b, ls, lc, level, B, offs, next);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        if (total == 0)
            break;
        lstart.push_back(next);
        lcount.push_back(total);
    }
    const int64_t nn = lstart.back() + lcount.back();
    s->nnodes = nn;
    s->maxlevel = (int)lstart.size() - 1;

    // ---- multipoles, deepest level first
    double *M, *S;
    TPM_CHECK(tmp.get(&M, nn, st));
    TPM_CHECK(tmp.get(&S, 3 * nn, st));
    for (int level = (int)lstart.size() - 1; level >= 0; level--) {
        int64_t lc = lcount[level];
        k_multipole<<<blocks_for(lc), kThreads, 0, st>>>(b, lstart[level], lc, s->perm, s->pos, s->mass, M, S);
        count_launch();
        TPM_CUDA(cudaGetLastError());
    }

    // ---- pre-order
    uint64_t *okey, *pkey;
    uint32_t *oval, *pre2bfs;
    TPM_CHECK(tmp.get(&okey, nn, st));
    TPM_CHECK(tmp.get(&pkey, nn, st));
    TPM_CHECK(tmp.get(&oval, nn, st));
    TPM_CHECK(tmp.get(&pre2bfs, nn, st));
    k_preorder_keys<<<blocks_for(nn), kThreads, 0, st>>>(b, nn, okey, oval);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    size_t sb2 = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sb2, okey, pkey, oval, pre2bfs, (int)nn, 0, 37, st));
    void *cub_tmp2 = cub_tmp;
    if (sb2 > cub_bytes)
        TPM_CHECK(tmp.get((char **)&cub_tmp2, sb2, st));
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp2, sb2, okey, pkey, oval, pre2bfs, (int)nn, 0, 37, st));
    count_cub_call();

    TPM_CHECK(s->mem.get(&s->ncen, nn, st));
    TPM_CHECK(s->mem.get(&s->ncom, nn, st));
    TPM_CHECK(s->mem.get(&s->nlink, nn, st));
    TPM_CHECK(s->mem.get(&s->nlevel, nn, st));
    TPM_CHECK(s->mem.get(&s->nprefix, nn, st));
    TPM_CHECK(s->mem.get(&s->nmass, nn, st));
    TPM_CHECK(s->mem.get(&s->ncomd, 3 * nn, st));
    NodeOut o{s->ncen, s->ncom, s->nlink, s->nlevel, s->nprefix, s->nmass, s->ncomd};
    k_finalize<<<blocks_for(nn), kThreads, 0, st>>>(b, pkey, pre2bfs, nn, M, S, s->x0[0], s->x0[1], s->x0[2], s->L0, o);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    k_leaf_particles<<<blocks_for(nn), kThreads, 0, st>>>(s->ncen, s->nlink, nn, s->perm, s->pos, s->mass, s->x0[0],
                                                          s->x0[1], s->x0[2], s->spart);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
