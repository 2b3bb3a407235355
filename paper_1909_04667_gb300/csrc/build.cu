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
//      its non-empty octants: eight threads per cell find the eight octant
//      boundaries in the sorted keys at once, and one atomic per cell
//      reserves its children (contiguous, in ascending octant order); the
//      level ranges stay on the device, so no host round trip is needed
//      between levels
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
    // warp-level min / max, then one atomic per block
    __shared__ long long red[2][3][32];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long l = have ? lo[a] : LLONG_MAX, h = have ? hi[a] : LLONG_MIN;
        for (int o = 16; o > 0; o >>= 1) {
            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][a][w] = l;
            red[1][a][w] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        long long l = LLONG_MAX, h = LLONG_MIN;
        for (int i = 0; i < nw; i++) {
            l = min(l, red[0][a][i]);
            h = max(h, red[1][a][i]);
        }
        atomicMin(&bbox[a], l);
        atomicMax(&bbox[3 + a], h);
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

// Device-side bookkeeping of one build.
struct BuildState {
    long long bbox[6];
    int bad;
    int overflow;
    unsigned total;  // nodes reserved so far
    int maxlevel;
    unsigned lstart[kMaxLevel + 2];
    unsigned lcount[kMaxLevel + 2];
    double x0[3];
    double L0;
    double scale;  // 2^21 / L0
};

__device__ double pow2_ceil_d(double x) {
    int e;
    const double f = frexp(x, &e);
    return (f == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// Root cube (one thread): periodic [0, box); open boundaries: the smallest
// power of two L0 >= 1.25 x the largest extent, x0 = lo - shift (L0 - extent)
// rounded down to the 2^-21 L0 grid.  Round-to-nearest operations only.
__global__ void k_root(BuildState *__restrict__ st, int periodic, double box, double s0, double s1, double s2) {
    if (threadIdx.x != 0)
        return;
    if (periodic) {
        st->x0[0] = st->x0[1] = st->x0[2] = 0.0;
        st->L0 = box;
    } else {
        double lo[3], hi[3], ext = 0.0;
        for (int a = 0; a < 3; a++) {
            lo[a] = from_ordered_bits(st->bbox[a]);
            hi[a] = from_ordered_bits(st->bbox[3 + a]);
            ext = fmax(ext, __dsub_rn(hi[a], lo[a]));
        }
        if (!(ext > 0.0))
            ext = 1.0;
        const double L0 = pow2_ceil_d(__dmul_rn(1.25, ext));
        const double unit = ldexp(L0, -kMaxLevel);
        const double sh[3] = {s0, s1, s2};
        for (int a = 0; a < 3; a++) {
            const double slack = __dsub_rn(L0, __dsub_rn(hi[a], lo[a]));
            const double x0 = __dsub_rn(lo[a], __dmul_rn(sh[a], slack));
            st->x0[a] = __dmul_rn(floor(__ddiv_rn(x0, unit)), unit);
        }
        st->L0 = L0;
    }
    st->scale = __ddiv_rn(ldexp(1.0, kMaxLevel), st->L0);
}

// K1: Morton keys of the 21-bit cell coordinates q = floor((x - x0) 2^21 / L0).
__global__ void k_keys(const double *__restrict__ pos, int64_t n, const BuildState *__restrict__ st,
                       uint64_t *__restrict__ key, uint32_t *__restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double o[3] = {st->x0[0], st->x0[1], st->x0[2]};
    const double scale = st->scale;
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
    uint32_t *first, *count, *child, *nchild, *parent, *arrive;
    uint8_t *level;
    uint64_t *prefix;
};

__global__ void k_level0(LevelArrays b, BuildState *__restrict__ st, int64_t n) {
    if (threadIdx.x != 0)
        return;
    b.first[0] = 0;
    b.count[0] = (uint32_t)n;
    b.level[0] = 0;
    b.prefix[0] = 0;
    b.parent[0] = 0;
    st->lstart[0] = 0;
    st->lcount[0] = 1;
}

// K3: splits every cell of one level that holds more than B particles (and is
// above the depth cap) into its non-empty octants.  Eight consecutive threads
// serve one cell: thread o finds where octant o starts in the cell's key
// range; the cell's first thread reserves the children with one atomic on
// the next level's counter.  Level l + 1 starts right after level l, whose
// size is final once the previous launch has finished.
__global__ void k_split_level(const uint64_t *__restrict__ key, LevelArrays b, BuildState *__restrict__ st, int level,
                              int bucket, unsigned cap) {
    // nodes past the node space (reserved after an overflow) were never written
    const unsigned ls = st->lstart[level], lc_all = st->lcount[level];
    const unsigned lc = ls >= cap ? 0u : min(lc_all, cap - ls);
    const unsigned next_start = ls + lc_all;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        st->lstart[level + 1] = next_start;
    const int lane = threadIdx.x & 31;
    const unsigned gmask = 0xffu << (lane & 24);
    const int o = lane & 7;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)lc * 8; t += stride) {
        const unsigned node = ls + (unsigned)(t >> 3);
        const uint32_t f = b.first[node], c = b.count[node];
        const bool split = (int)c > bucket && level < kMaxLevel;
        if (!split) {
            if (o == 0) {
                b.child[node] = 0;
                b.nchild[node] = 0;
            }
            continue;
        }
        const int shift = 3 * (kMaxLevel - level - 1);
        const uint64_t base = b.prefix[node] << 3;
        const uint32_t lo = (o == 0) ? f : lower_bound_key(key, f, f + c, (base | (uint64_t)o) << shift);
        uint32_t hi = __shfl_down_sync(gmask, lo, 1, 8);
        if (o == 7)
            hi = f + c;
        const bool nonempty = hi > lo;
        const unsigned bm = (__ballot_sync(gmask, nonempty) >> (lane & 24)) & 0xffu;
        const unsigned nch = __popc(bm);
        unsigned first_child = 0;
        if (o == 0)
            first_child = next_start + atomicAdd(&st->lcount[level + 1], nch);
        first_child = __shfl_sync(gmask, first_child, 0, 8);
        // out of node space: the host rebuilds with more.  The children that
        // still fit are written all the same, so that every slot below the
        // cap that the next level visits holds a valid key range.
        const bool fits = (uint64_t)first_child + nch <= cap;
        if (nonempty) {
            const unsigned ch = first_child + __popc(bm & ((1u << o) - 1u));
            if (ch < cap) {
                b.first[ch] = lo;
                b.count[ch] = hi - lo;
                b.level[ch] = (uint8_t)(level + 1);
                b.prefix[ch] = base | (uint64_t)o;
                b.parent[ch] = node;
            }
        }
        if (o == 0) {
            if (!fits)
                st->overflow = 1;
            b.child[node] = fits ? first_child : 0u;
            b.nchild[node] = fits ? nch : 0u;
        }
    }
}

// K4: FP64 monopoles in one pass, bottom-up.  Each leaf sums its particles in
// sorted order; then the last child of a node to finish (counted with an
// atomic on the parent) sums the node's children in ascending octant order,
// and so on up to the root.  Explicit round-to-nearest adds / muls, so every
// sum has the same fixed order and value whichever thread computes it.
__global__ void k_multipole(LevelArrays b, int64_t total, const uint32_t *__restrict__ perm,
                            const double *__restrict__ pos, const float *__restrict__ mass, double *__restrict__ M,
                            double *__restrict__ S) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= total || b.nchild[node] != 0)
        return;
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    const uint32_t f = b.first[node], e = f + b.count[node];
    for (uint32_t s = f; s < e; s++) {
        const uint32_t j = perm[s];
        const double mj = (double)mass[j];
        m = __dadd_rn(m, mj);
        sx = __dadd_rn(sx, __dmul_rn(mj, pos[3 * j]));
        sy = __dadd_rn(sy, __dmul_rn(mj, pos[3 * j + 1]));
        sz = __dadd_rn(sz, __dmul_rn(mj, pos[3 * j + 2]));
    }
    M[node] = m;
    S[3 * node] = sx;
    S[3 * node + 1] = sy;
    S[3 * node + 2] = sz;
    uint32_t cur = (uint32_t)node;
    while (cur != 0) {
        const uint32_t p = b.parent[cur];
        __threadfence();  // this node's sums are visible before the parent learns it is done
        const uint32_t nc = b.nchild[p];
        if (atomicAdd(&b.arrive[p], 1u) != nc - 1)
            return;  // a sibling still works; it will carry on upwards
        __threadfence();
        m = sx = sy = sz = 0.0;
        const uint32_t c0 = b.child[p];
        for (uint32_t c = c0; c < c0 + nc; c++) {
            m = __dadd_rn(m, __ldcg(&M[c]));
            sx = __dadd_rn(sx, __ldcg(&S[3 * c]));
            sy = __dadd_rn(sy, __ldcg(&S[3 * c + 1]));
            sz = __dadd_rn(sz, __ldcg(&S[3 * c + 2]));
        }
        M[p] = m;
        S[3 * p] = sx;
        S[3 * p + 1] = sy;
        S[3 * p + 2] = sz;
        cur = p;
    }
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

// Breadth-first node records for the group walk (same values as the pre-order
// tables; children of a node are contiguous in this order).
__global__ void k_finalize_bfs(LevelArrays b, int64_t total, const double *__restrict__ M,
                               const double *__restrict__ S, double x0, double y0, double z0, double L0,
                               float4 *__restrict__ bcen, float4 *__restrict__ bcom, int4 *__restrict__ blink) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total)
        return;
    const int lvl = b.level[i];
    const uint64_t pre = b.prefix[i];
    const double m = M[i];
    const double cx = __ddiv_rn(S[3 * i], m), cy = __ddiv_rn(S[3 * i + 1], m), cz = __ddiv_rn(S[3 * i + 2], m);
    const double half = ldexp(L0, -(lvl + 1));
    const double rx = (double)(2 * (uint64_t)compact3(pre) + 1) * half;
    const double ry = (double)(2 * (uint64_t)compact3(pre >> 1) + 1) * half;
    const double rz = (double)(2 * (uint64_t)compact3(pre >> 2) + 1) * half;
    bcen[i] = make_float4((float)rx, (float)ry, (float)rz, (float)(2.0 * half));
    bcom[i] = make_float4((float)__dsub_rn(cx, __dadd_rn(x0, rx)), (float)__dsub_rn(cy, __dadd_rn(y0, ry)),
                          (float)__dsub_rn(cz, __dadd_rn(z0, rz)), (float)m);
    blink[i] = make_int4((int)b.child[i], (int)b.nchild[i], (int)b.first[i], (int)b.count[i]);
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
    TPM_CHECK(s->mem.get(&s->err, 1, st));
    TPM_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));

    BuildState *dst;
    TPM_CHECK(tmp.get(&dst, 1, st));
    // the context's pinned page holds the host copy of the build state; one
    // build at a time per context uses it
    static_assert(sizeof(BuildState) <= kPinnedStateBytes, "build state exceeds the pinned page");
    std::lock_guard<std::mutex> build_lock(c->build_mu);
    BuildState *hst = static_cast<BuildState *>(c->pinned_state);
    memset(hst, 0, sizeof(BuildState));
    for (int a = 0; a < 3; a++) {
        hst->bbox[a] = LLONG_MAX;
        hst->bbox[3 + a] = LLONG_MIN;
    }
    TPM_CUDA(cudaMemcpyAsync(dst, hst, sizeof(BuildState), cudaMemcpyHostToDevice, st));
    const unsigned grid = (unsigned)(c->num_sms * 8);

    // ---- prepare, bounding box, root, keys, sort
    k_prepare<<<blocks_for(n), kThreads, 0, st>>>(pos_in, mass_in, n, s->bp.periodic, s->bp.box, s->bp.shift[0],
                                                   s->bp.shift[1], s->bp.shift[2], s->pos, s->mass, dst->bbox,
                                                   &dst->bad);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    k_root<<<1, 32, 0, st>>>(dst, s->bp.periodic, s->bp.box, s->bp.shift[0], s->bp.shift[1], s->bp.shift[2]);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    uint64_t *key_raw;
    uint32_t *idx_raw;
    TPM_CHECK(tmp.get(&key_raw, n, st));
    TPM_CHECK(tmp.get(&idx_raw, n, st));
    k_keys<<<blocks_for(n), kThreads, 0, st>>>(s->pos, n, dst, key_raw, idx_raw);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    size_t sort_bytes = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, key_raw, s->key, idx_raw, s->perm, (int)n, 0,
                                             3 * kMaxLevel, st));
    void *cub_tmp;
    TPM_CHECK(tmp.get((char **)&cub_tmp, sort_bytes, st));
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp, sort_bytes, key_raw, s->key, idx_raw, s->perm, (int)n, 0,
                                             3 * kMaxLevel, st));
    count_cub_call();
    k_rank<<<blocks_for(n), kThreads, 0, st>>>(s->perm, n, s->rank);
    count_launch();
    TPM_CUDA(cudaGetLastError());

    // ---- levels and monopoles, all on the device; retried with more node
    // space in the rare case the first guess is too small
    // node space: ~0.4 n nodes for B = 8, ~1.5 n for B = 1; an overflow retries
    unsigned cap = (unsigned)std::min<int64_t>((B == 1 ? 2 * n : n) + 1024, 0x7fffffffLL);
    LevelArrays b{};
    double *M = nullptr, *S = nullptr;
    AllocSet lv;
    lv.ctx = c;
    struct LvGuard {
        AllocSet &t;
        cudaStream_t st;
        ~LvGuard() { t.release(st); }
    } lguard{lv, st};
    for (int attempt = 0;; attempt++) {
        lv.release(st);
        TPM_CHECK(lv.get(&b.first, cap, st));
        TPM_CHECK(lv.get(&b.count, cap, st));
        TPM_CHECK(lv.get(&b.child, cap, st));
        TPM_CHECK(lv.get(&b.nchild, cap, st));
        TPM_CHECK(lv.get(&b.level, cap, st));
        TPM_CHECK(lv.get(&b.prefix, cap, st));
        TPM_CHECK(lv.get(&b.parent, cap, st));
        TPM_CHECK(lv.get(&b.arrive, cap, st));
        TPM_CHECK(lv.get(&M, cap, st));
        TPM_CHECK(lv.get(&S, 3 * (size_t)cap, st));
        TPM_CUDA(cudaMemsetAsync(&dst->overflow, 0, sizeof(int), st));
        TPM_CUDA(cudaMemsetAsync(dst->lcount, 0, sizeof(dst->lcount), st));
        TPM_CUDA(cudaMemsetAsync(b.arrive, 0, (size_t)cap * sizeof(uint32_t), st));
        k_level0<<<1, 32, 0, st>>>(b, dst, n);
        count_launch();
        for (int level = 0; level <= kMaxLevel; level++) {
            k_split_level<<<grid, kThreads, 0, st>>>(s->key, b, dst, level, B, cap);
            count_launch();
        }
        TPM_CUDA(cudaGetLastError());
        TPM_CUDA(cudaMemcpyAsync(hst, dst, sizeof(BuildState), cudaMemcpyDeviceToHost, st));
        TPM_CUDA(cudaStreamSynchronize(st));
        if (hst->bad & 1) {
            set_error("non-finite position");
            return TPM_ENAN;
        }
        if (hst->bad & 4) {
            set_error("masses must be finite and > 0");
            return TPM_ENAN;
        }
        if (hst->bad & 2) {
            set_error("periodic positions must lie in [0, box)");
            return TPM_EINVAL;
        }
        uint64_t total = 0;
        int maxlevel = 0;
        for (int l = 0; l <= kMaxLevel; l++) {
            total += hst->lcount[l];
            if (hst->lcount[l])
                maxlevel = l;
        }
        if (!hst->overflow) {
            hst->total = (unsigned)total;
            hst->maxlevel = maxlevel;
            break;
        }
        // the count seen is a lower bound (subtrees below the cap's edge were
        // not explored); no level holds more than min(8^l, n) nodes
        uint64_t bound = 0;
        for (int l = 0; l <= kMaxLevel; l++)
            bound += std::min<uint64_t>(l < 21 ? uint64_t(1) << (3 * l) : UINT64_MAX, (uint64_t)n);
        bound = std::min<uint64_t>(bound, 0x7fffffffULL);
        if (attempt >= 5 || cap >= bound) {
            set_error("tree node space overflow (at least %llu nodes needed)", (unsigned long long)total);
            return TPM_ECUDA;
        }
        cap = (unsigned)std::min<uint64_t>(std::max<uint64_t>(4 * total, 2 * (uint64_t)cap) + 1024, bound);
    }
    for (int a = 0; a < 3; a++)
        s->x0[a] = hst->x0[a];
    s->L0 = hst->L0;
    const int64_t nn = hst->total;
    s->nnodes = nn;
    s->maxlevel = hst->maxlevel;

    // ---- monopoles, bottom-up in one pass
    k_multipole<<<blocks_for(nn), kThreads, 0, st>>>(b, nn, s->perm, s->pos, s->mass, M, S);
    count_launch();
    TPM_CUDA(cudaGetLastError());

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
    if (sb2 > sort_bytes)
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
    TPM_CHECK(s->mem.get(&s->bcen, nn, st));
    TPM_CHECK(s->mem.get(&s->bcom, nn, st));
    TPM_CHECK(s->mem.get(&s->blink, nn, st));
    k_finalize_bfs<<<blocks_for(nn), kThreads, 0, st>>>(b, nn, M, S, s->x0[0], s->x0[1], s->x0[2], s->L0, s->bcen,
                                                        s->bcom, s->blink);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    k_leaf_particles<<<blocks_for(nn), kThreads, 0, st>>>(s->ncen, s->nlink, nn, s->perm, s->pos, s->mass, s->x0[0],
                                                          s->x0[1], s->x0[2], s->spart);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
