// Oct-tree construction on the GPU (paper Sec. 3.1).
//
// The paper inserts particles one at a time and splits every leaf that would
// hold two of them.  The cells that exist at the end do not depend on the
// insertion order -- a cell exists when its parent holds more than the leaf
// bucket B -- so the same tree is built here in parallel from sorted keys:
//
//   1. root cube and 21-bit integer cell coordinates -> 63-bit Morton keys
//   2. stable radix sort of (key, particle index)
//   3. the nodes straight from the sorted keys, in depth-first pre-order:
//      with w(j) the deepest level shared by keys j and j + B, the cell
//      around particle i holds more than B particles down to level
//      max w(j) over j in [i - B, i], so i's leaf level D(i) is one below
//      (capped at 21); the nodes whose first particle is i are its cells at
//      the levels below the level it shares with particle i - 1, down to
//      D(i).  Nodes ordered by (first particle, level) are the pre-order,
//      so a scan of the per-particle node counts places every node; particle
//      ranges, skip indices and parents follow from searches in the sorted
//      keys.  No level-by-level passes and no host round trip but one (the
//      node count, to size the node tables)
//   4. FP64 masses and mass-weighted positions summed bottom-up in one pass,
//      children in ascending octant order and a leaf's particles in sorted
//      order, with explicit round-to-nearest operations (no contraction), so
//      the result is the same bit for bit on any correct implementation of
//      that order
//   5. pre-order and breadth-first tables for the walks: per node the FP32 geometric
//      centre (exact: it lies on the 2^-22 L0 grid), side, centre of mass
//      relative to the centre, mass, skip index, particle range and leaf flag
//      -- three 16-byte records loaded with one vector load each -- and per
//      sorted particle its position relative to its leaf centre plus mass.
#include <cub/cub.cuh>
#include <cuda/atomic>

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

// Device-side bookkeeping of one build (its host copy also receives the node
// count).
struct BuildState {
    long long bbox[6];
    int bad;
    unsigned total;  // nodes of the tree
    double x0[3];
    double L0;
    double scale;  // 2^21 / L0
    unsigned blocks_done;  // k_prepare blocks that have reduced their bounding box
};

__device__ double pow2_ceil_d(double x) {
    int e;
    const double f = frexp(x, &e);
    return (f == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// Root cube (one thread, once the bounding box is complete): periodic
// [0, box); open boundaries: the smallest power of two L0 >= 1.25 x the
// largest extent, x0 = lo - shift (L0 - extent) rounded down to the 2^-21 L0
// grid.  Round-to-nearest operations only.
__device__ void root_cube(BuildState *__restrict__ st, int periodic, double box, double s0, double s1, double s2) {
    if (periodic) {
        st->x0[0] = st->x0[1] = st->x0[2] = 0.0;
        st->L0 = box;
    } else {
        double lo[3], hi[3], ext = 0.0;
        for (int a = 0; a < 3; a++) {
            lo[a] = from_ordered_bits(__ldcg(&st->bbox[a]));  // reduced by other blocks' atomics
            hi[a] = from_ordered_bits(__ldcg(&st->bbox[3 + a]));
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

// Copies positions and masses into the system, applies the periodic shift and
// wrap, checks finiteness and ranges (and the per-particle softening lengths,
// if any), and reduces the bounding box; the last block to finish computes the
// root cube from it.
__global__ void k_prepare(const double *__restrict__ pin, const float *__restrict__ mass_in,
                          const float *__restrict__ hsoft, int64_t n, int periodic, double box, double s0, double s1,
                          double s2, double *__restrict__ pout, float *__restrict__ mout,
                          BuildState *__restrict__ state) {
    long long *bbox = state->bbox;
    int *bad = &state->bad;
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
        if (hsoft) {
            const float h = hsoft[i];
            if (!(h > 0.0f) || !isfinite(h))
                atomicOr(bad, 8);
        }
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
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&state->blocks_done, 1u) == gridDim.x - 1) {
        __threadfence();
        root_cube(state, periodic, box, s0, s1, s2);
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

// floor(v) clamped to [0, 2^21 - 1], read off the bits of v (integer
// operations only: FP64 arithmetic is scarce on this GPU).  v = m 2^(e - 52)
// with the 53-bit significand m; for 1 <= v < 2^21 the integer part is
// m >> (52 - e); negative v (sign bit set) and v < 1 give 0, v >= 2^21 (and
// non-finite v) the largest coordinate.
__device__ __forceinline__ uint32_t cell_coord(double v) {
    const long long b = __double_as_longlong(v);
    if (b < 0)
        return 0u;
    const int e = (int)(b >> 52) - 1023;
    if (e < 0)
        return 0u;
    if (e >= kMaxLevel)
        return (1u << kMaxLevel) - 1u;
    const uint64_t m = ((uint64_t)b & 0xfffffffffffffull) | (1ull << 52);
    return (uint32_t)(m >> (52 - e));
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
    for (int a = 0; a < 3; a++)
        k |= spread3(cell_coord(__dmul_rn(__dsub_rn(pos[3 * i + a], o[a]), scale))) << a;
    key[i] = k;
    idx[i] = (uint32_t)i;
}

// Inverse permutation, and positions and masses gathered into key order for
// the passes over leaves.
__global__ void k_rank(const uint32_t *__restrict__ perm, int64_t n, const double *__restrict__ pos,
                       const float *__restrict__ mass, const float *__restrict__ hsoft, uint32_t *__restrict__ rank,
                       double *__restrict__ spos, float *__restrict__ smass, float *__restrict__ psoft) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    const uint32_t j = perm[s];
    rank[j] = (uint32_t)s;
    spos[3 * s] = pos[3 * j];
    spos[3 * s + 1] = pos[3 * j + 1];
    spos[3 * s + 2] = pos[3 * j + 2];
    smass[s] = mass[j];
    if (hsoft)  // per-particle softening, in key order (checked by k_prepare)
        psoft[s] = hsoft[j];
}

// Deepest level whose cell holds both keys (kMaxLevel when they are equal).
__device__ __forceinline__ int common_level(uint64_t a, uint64_t b) {
    const uint64_t x = a ^ b;
    return x ? (kMaxLevel - 1) - (63 - __clzll((long long)x)) / 3 : kMaxLevel;
}

// Smallest e in [lo, hi] with e == hi or key[e] >= bound (keys ascending,
// key[lo - 1] < bound): exponential search from lo, then bisection.
__device__ __forceinline__ uint32_t search_up(const uint64_t *__restrict__ key, uint32_t lo, uint32_t hi,
                                              uint64_t bound) {
    uint32_t a = lo, b = lo;
    uint64_t step = 1;
    while (b < hi && key[b] < bound) {
        a = b + 1;
        b = (uint64_t)(hi - b) > step ? b + (uint32_t)step : hi;
        step <<= 1;
    }
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (key[mid] < bound)
            a = mid + 1;
        else
            b = mid;
    }
    return a;
}

// Smallest f <= i with key[f] >= bound, given key[i] >= bound: exponential
// search downwards from i, then bisection.
__device__ __forceinline__ uint32_t search_down(const uint64_t *__restrict__ key, uint32_t i, uint64_t bound) {
    int64_t hi = i, lo = (int64_t)i - 1, step = 1;
    while (lo >= 0 && key[lo] >= bound) {
        hi = lo;
        lo -= step;
        step <<= 1;
    }
    int64_t a = lo + 1 > 0 ? lo + 1 : 0, b = hi;
    while (a < b) {
        const int64_t mid = a + ((b - a) >> 1);
        if (key[mid] < bound)
            a = mid + 1;
        else
            b = mid;
    }
    return (uint32_t)a;
}

// K3a. Which cells hold more than B particles.  The level-m cell around sorted
// particle i holds more than B particles iff some run of B + 1 consecutive
// particles inside it contains i, i.e. iff w(j) >= m for some j in [i - B, i],
// where w(j) = common_level(key[j], key[j + B]).  The window maximum over
// [i - B, i] comes from prefix and suffix maxima inside blocks of B + 1
// entries (one thread per block); this kernel writes them.
__global__ void k_window_max(const uint64_t *__restrict__ key, int64_t n, int B, int8_t *__restrict__ pre_max,
                             int8_t *__restrict__ suf_max) {
    const int64_t W = (int64_t)B + 1;
    const int64_t j0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * W;
    if (j0 >= n)
        return;
    const int64_t j1 = min(j0 + W, n);
    int m = -1;
    for (int64_t j = j0; j < j1; j++) {
        const int w = j + B < n ? common_level(key[j], key[j + B]) : -1;
        suf_max[j] = (int8_t)w;
        m = max(m, w);
        pre_max[j] = (int8_t)m;
    }
    m = -1;
    for (int64_t j = j1 - 1; j >= j0; j--) {
        m = max(m, (int)suf_max[j]);
        suf_max[j] = (int8_t)m;
    }
}

// K3b. Per sorted particle i: the level of its leaf, D(i) = min(1 + deepest
// level whose cell around i holds more than B particles, 21), and the levels
// at which i is the first particle of its cell, (common_level(key[i-1],
// key[i]), D(i)].  Those cells are exactly the nodes whose first particle is
// i, and ordering all nodes by (first particle, level) is the depth-first
// pre-order: an exclusive scan of the per-particle counts gives every node
// its pre-order index directly.
__global__ void k_node_counts(const uint64_t *__restrict__ key, int64_t n, int B, const int8_t *__restrict__ pre_max,
                              const int8_t *__restrict__ suf_max, uint8_t *__restrict__ top_level,
                              uint8_t *__restrict__ leaf_level, uint32_t *__restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int lp = i ? common_level(key[i - 1], key[i]) : -1;
    int split = pre_max[i];  // deepest level whose cell around i holds > B particles
    if (i - B >= 0)
        split = max(split, (int)suf_max[i - B]);
    const int D = min(split + 1, kMaxLevel);
    top_level[i] = (uint8_t)(lp + 1);
    leaf_level[i] = (uint8_t)D;
    cnt[i] = (uint32_t)max(D - lp, 0);
}

// Pre-order node arrays of the build.
struct NodeArrays {
    uint32_t *first, *count, *skip, *parent, *nchild, *arrive, *order;
    uint8_t *level;
    uint64_t *prefix;
};

// K3c. The nodes whose first particle is sorted particle i, from the top
// down: particle range (the cell's end found by searching the sorted keys),
// skip index (the first node of the particle just past the cell), key prefix,
// parent (the node above with the same first particle, else the cell found by
// searching downwards) and, by one atomic per node, the parent's child count.
__global__ void k_nodes(const uint64_t *__restrict__ key, int64_t n, const uint32_t *__restrict__ base,
                        const uint8_t *__restrict__ top_level, const uint8_t *__restrict__ leaf_level, NodeArrays t) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint32_t p0 = base[i], nc = base[i + 1] - p0;
    if (nc == 0)
        return;
    const uint32_t total = base[n];
    const int l0 = top_level[i];
    const uint64_t ki = key[i];
    uint32_t end = (uint32_t)n;
    for (uint32_t k = 0; k < nc; k++) {
        const int l = l0 + (int)k;
        const uint32_t p = p0 + k;
        const int sh = 3 * (kMaxLevel - l);
        const uint64_t pre = ki >> sh;
        end = search_up(key, (uint32_t)i + 1, end, (pre + 1) << sh);  // cells nest: the end only shrinks
        t.first[p] = (uint32_t)i;
        t.count[p] = end - (uint32_t)i;
        t.skip[p] = end < n ? base[end] : total;
        t.level[p] = (uint8_t)l;
        t.prefix[p] = pre;
        t.order[p] = p;
        uint32_t par = 0;
        if (l > 0) {
            if (k > 0) {
                par = p - 1;
            } else {
                const uint32_t f = search_down(key, (uint32_t)i, (pre >> 3) << (sh + 3));
                par = base[f] + (uint32_t)(l - 1 - top_level[f]);
            }
            atomicAdd(&t.nchild[par], 1u);
        }
        t.parent[p] = par;
    }
}

// K4: FP64 monopoles in one pass, bottom-up.  Each leaf sums its particles in
// sorted order; then the last child of a node to finish (counted with an
// atomic on the parent) sums the node's children in ascending octant order,
// and so on up to the root.  Sums are stored by breadth-first index, where a
// node's children are contiguous, so the children's sums load independently.
// Explicit round-to-nearest adds / muls, so every sum has the same fixed
// order and value whichever thread computes it.  The climb is a chain of
// dependent memory round trips, so each step loads the links it needs next
// (parent, child count, breadth-first indices: read-only here) before its
// atomic, and a leaf loads its particles four at a time before summing them.
__global__ void k_multipole(NodeArrays t, int64_t total, const uint32_t *__restrict__ pre2bfs,
                            const double *__restrict__ spos, const float *__restrict__ smass, double *__restrict__ M,
                            double *__restrict__ S, const float *__restrict__ psoft, float *__restrict__ hmx,
                            float *__restrict__ hmn) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= total || t.nchild[node] != 0)
        return;
    const uint32_t f = t.first[node], e = f + t.count[node];
    uint32_t p = node ? t.parent[node] : 0u;  // the climb's first parent
    uint32_t q = pre2bfs[node];
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    float hi = 0.0f, lo = INFINITY;  // largest / smallest softening (per-particle softening only)
    for (uint32_t s = f; s < e; s += 4) {
        double ms[4], px[4], py[4], pz[4];
        float hs[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t j = min(s + u, e - 1);
            ms[u] = (double)smass[j];
            px[u] = spos[3 * j];
            py[u] = spos[3 * j + 1];
            pz[u] = spos[3 * j + 2];
            hs[u] = psoft ? psoft[j] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (s + u < e) {
                m = __dadd_rn(m, ms[u]);
                sx = __dadd_rn(sx, __dmul_rn(ms[u], px[u]));
                sy = __dadd_rn(sy, __dmul_rn(ms[u], py[u]));
                sz = __dadd_rn(sz, __dmul_rn(ms[u], pz[u]));
                if (psoft) {
                    hi = fmaxf(hi, hs[u]);
                    lo = fminf(lo, hs[u]);
                }
            }
        }
    }
    M[q] = m;
    S[3 * q] = sx;
    S[3 * q + 1] = sy;
    S[3 * q + 2] = sz;
    if (psoft) {
        hmx[q] = hi;
        hmn[q] = lo;
    }
    uint32_t cur = (uint32_t)node;
    while (cur != 0) {
        // links of this step, loaded ahead of the atomic
        const uint32_t nc = t.nchild[p];
        const uint32_t c0 = pre2bfs[p + 1];  // first child; the others follow it
        const uint32_t pq = pre2bfs[p];
        const uint32_t pp = p ? t.parent[p] : 0u;
        // release: this node's sums are visible before the parent learns it is
        // done; acquire: the last child sees all its siblings' sums
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device> arrive(t.arrive[p]);
        if (arrive.fetch_add(1u, cuda::memory_order_acq_rel) != nc - 1)
            return;  // a sibling still works; it will carry on upwards
        m = sx = sy = sz = 0.0;
        hi = 0.0f;
        lo = INFINITY;
        for (uint32_t c = c0; c < c0 + nc; c++) {
            m = __dadd_rn(m, __ldcg(&M[c]));
            sx = __dadd_rn(sx, __ldcg(&S[3 * c]));
            sy = __dadd_rn(sy, __ldcg(&S[3 * c + 1]));
            sz = __dadd_rn(sz, __ldcg(&S[3 * c + 2]));
            if (psoft) {
                hi = fmaxf(hi, __ldcg(&hmx[c]));
                lo = fminf(lo, __ldcg(&hmn[c]));
            }
        }
        M[pq] = m;
        S[3 * pq] = sx;
        S[3 * pq + 1] = sy;
        S[3 * pq + 2] = sz;
        if (psoft) {
            hmx[pq] = hi;
            hmn[pq] = lo;
        }
        cur = p;
        p = pp;
    }
}

// Inverse of the breadth-first -> pre-order map.
__global__ void k_invert(const uint32_t *__restrict__ bfs2pre, int64_t total, uint32_t *__restrict__ pre2bfs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < total)
        pre2bfs[bfs2pre[q]] = (uint32_t)q;
}

struct NodeOut {
    float4 *cen, *com;
    int4 *link;
    uint8_t *level;
    uint64_t *prefix;
    float4 *bcen, *bcom;
    int4 *blink;
    float4 *spart;
    float *nsoft, *bsoft;  // per-particle softening only
};

// Exact centre of node (lvl, pre) relative to x0: (2 i + 1) L0 2^-(lvl + 1)
// per axis, i the cell index along the axis read off the key prefix; the
// power of two is built from its bits (exact scaling, lvl <= 21).
struct NodeGeom {
    double rx, ry, rz, side;
};
__device__ __forceinline__ NodeGeom node_geom(uint64_t pre, int lvl, double L0) {
    const double half = __dmul_rn(L0, __longlong_as_double((long long)(1022 - lvl) << 52));
    NodeGeom g;
    g.rx = __dmul_rn((double)(2 * (uint64_t)compact3(pre) + 1), half);
    g.ry = __dmul_rn((double)(2 * (uint64_t)compact3(pre >> 1) + 1), half);
    g.rz = __dmul_rn((double)(2 * (uint64_t)compact3(pre >> 2) + 1), half);
    g.side = 2.0 * half;
    return g;
}

// K5a: walk tables that do not need the monopoles, written while the monopole
// pass climbs.  Pre-order: FP32 geometric centre (exact, on the 2^-22 L0 grid)
// and side, (skip, first particle, count, leaf flag), level and key prefix
// for export; breadth-first: centre and (first child, child count, first
// particle, particle count); and every leaf's particles relative to the FP32
// leaf centre (FP64 difference rounded to FP32) with their masses.
__global__ void k_tables(NodeArrays t, const uint32_t *__restrict__ pre2bfs, int64_t total,
                         const double *__restrict__ spos, const float *__restrict__ smass, double x0, double y0,
                         double z0, double L0, NodeOut o) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= total)
        return;
    const uint32_t f = t.first[p], c = t.count[p], nch = t.nchild[p];
    const int lvl = t.level[p];
    const uint64_t pre = t.prefix[p];
    const uint32_t q = pre2bfs[p];
    const NodeGeom g = node_geom(pre, lvl, L0);
    const float4 cen = make_float4((float)g.rx, (float)g.ry, (float)g.rz, (float)g.side);
    o.cen[p] = cen;
    o.link[p] = make_int4((int)t.skip[p], (int)f, (int)c, nch == 0);
    o.level[p] = (uint8_t)lvl;
    o.prefix[p] = pre;
    o.bcen[q] = cen;
    o.blink[q] = make_int4(nch ? (int)pre2bfs[p + 1] : 0, (int)nch, (int)f, (int)c);
    if (nch == 0) {
        const double ax = __dadd_rn(x0, (double)cen.x), ay = __dadd_rn(y0, (double)cen.y),
                     az = __dadd_rn(z0, (double)cen.z);
        for (uint32_t s = f; s < f + c; s++)
            o.spart[s] = make_float4((float)__dsub_rn(spos[3 * s], ax), (float)__dsub_rn(spos[3 * s + 1], ay),
                                     (float)__dsub_rn(spos[3 * s + 2], az), smass[s]);
    }
}

// K5b: centre of mass relative to the exact geometric centre (FP32) and mass,
// pre-order and breadth-first, and the largest softening per node (negative
// when the node mixes softenings).  S / m is S times the correctly rounded
// 1 / m: one FP64 reciprocal instead of three divisions; the FP64 product is
// within an ulp of the quotient, far below the FP32 rounding of the offset.
__global__ void k_com(NodeArrays t, const uint32_t *__restrict__ pre2bfs, int64_t total,
                      const double *__restrict__ M, const double *__restrict__ S, const float *__restrict__ hmx,
                      const float *__restrict__ hmn, double x0, double y0, double z0, double L0, NodeOut o) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= total)
        return;
    const uint32_t q = pre2bfs[p];
    const NodeGeom g = node_geom(t.prefix[p], t.level[p], L0);
    const double m = M[q];
    const double rm = __drcp_rn(m);
    const double cx = __dmul_rn(S[3 * q], rm), cy = __dmul_rn(S[3 * q + 1], rm), cz = __dmul_rn(S[3 * q + 2], rm);
    const float4 com = make_float4((float)__dsub_rn(cx, __dadd_rn(x0, g.rx)), (float)__dsub_rn(cy, __dadd_rn(y0, g.ry)),
                                   (float)__dsub_rn(cz, __dadd_rn(z0, g.rz)), (float)m);
    o.com[p] = com;
    o.bcom[q] = com;
    if (hmx) {
        const float v = hmn[q] < hmx[q] ? -hmx[q] : hmx[q];
        o.nsoft[p] = v;
        o.bsoft[q] = v;
    }
}

}  // namespace

int build_tree_device(Ctx *c, System *s, const double *pos_in, const float *mass_in, const float *hsoft_in,
                      cudaStream_t st) {
    const int64_t n = s->n;
    const int B = s->bp.leaf_bucket;
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};

    // ---- memory for the particle passes: the system's arrays in one block,
    // the build's scratch in another (the CUB scratch sized for the key sort
    // and the node-count scan, whichever is larger)
    size_t sort_bytes = 0, scan_bytes = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                             (const uint32_t *)nullptr, (uint32_t *)nullptr, (int)n, 0, 3 * kMaxLevel,
                                             st));
    TPM_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                           (int)(n + 1), st));
    const size_t cub_bytes = std::max(sort_bytes, scan_bytes);
    Carve sys_a;
    sys_a.add(&s->pos, 3 * n);
    sys_a.add(&s->mass, n);
    sys_a.add(&s->key, n);
    sys_a.add(&s->perm, n);
    sys_a.add(&s->rank, n);
    sys_a.add(&s->spart, n);
    sys_a.add(&s->err, 1);
    if (hsoft_in)
        sys_a.add(&s->psoft, n);
    TPM_CHECK(sys_a.commit(s->mem, st));
    BuildState *dst;
    uint64_t *key_raw;
    uint32_t *idx_raw;
    char *cub_tmp;
    double *spos;
    float *smass;
    int8_t *pre_max, *suf_max;
    uint8_t *top_level, *leaf_level;
    uint32_t *cnt, *base;
    Carve tmp_a;
    tmp_a.add(&dst, 1);
    tmp_a.add(&key_raw, n);
    tmp_a.add(&idx_raw, n);
    tmp_a.add(&cub_tmp, cub_bytes);
    tmp_a.add(&spos, 3 * n);
    tmp_a.add(&smass, n);
    tmp_a.add(&pre_max, n);
    tmp_a.add(&suf_max, n);
    tmp_a.add(&top_level, n);
    tmp_a.add(&leaf_level, n);
    tmp_a.add(&cnt, n + 1);
    tmp_a.add(&base, n + 1);
    TPM_CHECK(tmp_a.commit(tmp, st));
    TPM_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));

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

    // ---- prepare, bounding box and root (last block), keys, sort
    k_prepare<<<blocks_for(n), kThreads, 0, st>>>(pos_in, mass_in, hsoft_in, n, s->bp.periodic, s->bp.box,
                                                   s->bp.shift[0], s->bp.shift[1], s->bp.shift[2], s->pos, s->mass,
                                                   dst);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    k_keys<<<blocks_for(n), kThreads, 0, st>>>(s->pos, n, dst, key_raw, idx_raw);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp, sort_bytes, key_raw, s->key, idx_raw, s->perm, (int)n, 0,
                                             3 * kMaxLevel, st));
    count_cub_call();

    // ---- node counts per particle and their scan: the pre-order indices
    k_window_max<<<blocks_for((n + B) / ((int64_t)B + 1)), kThreads, 0, st>>>(s->key, n, B, pre_max, suf_max);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(uint32_t), st));
    k_node_counts<<<blocks_for(n), kThreads, 0, st>>>(s->key, n, B, pre_max, suf_max, top_level, leaf_level, cnt);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cub::DeviceScan::ExclusiveSum(cub_tmp, scan_bytes, cnt, base, (int)(n + 1), st));
    count_cub_call();
    TPM_CUDA(cudaMemcpyAsync(hst, dst, sizeof(BuildState), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaMemcpyAsync(&hst->total, base + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaEventRecord(c->ev_state, st));
    // the particles gathered into key order while the host reads the state
    k_rank<<<blocks_for(n), kThreads, 0, st>>>(s->perm, n, s->pos, s->mass, hsoft_in, s->rank, spos, smass, s->psoft);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cudaEventSynchronize(c->ev_state));
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
    if (hst->bad & 8) {
        set_error("softening lengths must be finite and > 0");
        return TPM_ENAN;
    }
    for (int a = 0; a < 3; a++) {
        s->x0[a] = hst->x0[a];
        s->bb_lo[a] = from_ordered_bits(hst->bbox[a]);
        s->bb_hi[a] = from_ordered_bits(hst->bbox[3 + a]);
    }
    s->L0 = hst->L0;
    const int64_t nn = hst->total;
    s->nnodes = nn;

    // ---- memory for the node passes: scratch in one block, the system's
    // node tables in another
    NodeArrays t{};
    uint8_t *level_sorted;
    uint32_t *bfs2pre;
    float *hmx = nullptr, *hmn = nullptr;
    size_t lsort_bytes = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, lsort_bytes, (const uint8_t *)nullptr, (uint8_t *)nullptr,
                                             (const uint32_t *)nullptr, (uint32_t *)nullptr, (int)nn, 0, 5, st));
    char *lsort_tmp = cub_tmp;
    Carve tmp_b;
    // nchild and arrive adjacent: one memset clears both
    tmp_b.add(&t.nchild, nn);
    tmp_b.add(&t.arrive, nn);
    tmp_b.add(&t.first, nn);
    tmp_b.add(&t.count, nn);
    tmp_b.add(&t.skip, nn);
    tmp_b.add(&t.parent, nn);
    tmp_b.add(&t.order, nn);
    tmp_b.add(&t.level, nn);
    tmp_b.add(&t.prefix, nn);
    tmp_b.add(&level_sorted, nn);
    tmp_b.add(&bfs2pre, nn);
    if (lsort_bytes > cub_bytes)
        tmp_b.add(&lsort_tmp, lsort_bytes);
    if (s->psoft) {
        tmp_b.add(&hmx, nn);
        tmp_b.add(&hmn, nn);
    }
    TPM_CHECK(tmp_b.commit(tmp, st));
    Carve sys_b;
    sys_b.add(&s->msum, nn);  // FP64 sums by breadth-first index, kept with the system for export
    sys_b.add(&s->ssum, 3 * nn);
    sys_b.add(&s->pre2bfs, nn);
    sys_b.add(&s->ncen, nn);
    sys_b.add(&s->ncom, nn);
    sys_b.add(&s->nlink, nn);
    sys_b.add(&s->nlevel, nn);
    sys_b.add(&s->nprefix, nn);
    sys_b.add(&s->bcen, nn);
    sys_b.add(&s->bcom, nn);
    sys_b.add(&s->blink, nn);
    if (s->psoft) {
        sys_b.add(&s->nsoft, nn);
        sys_b.add(&s->bsoft, nn);
    }
    TPM_CHECK(sys_b.commit(s->mem, st));
    double *M = s->msum, *S = s->ssum;
    uint32_t *pre2bfs = s->pre2bfs;

    // ---- nodes in pre-order
    TPM_CUDA(cudaMemsetAsync(t.nchild, 0, (size_t)((char *)t.arrive - (char *)t.nchild) + nn * sizeof(uint32_t), st));
    k_nodes<<<blocks_for(n), kThreads, 0, st>>>(s->key, n, base, top_level, leaf_level, t);
    count_launch();
    TPM_CUDA(cudaGetLastError());

    // ---- breadth-first order: a stable sort of the pre-order by level
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(lsort_tmp, lsort_bytes, t.level, level_sorted, t.order, bfs2pre,
                                             (int)nn, 0, 5, st));
    count_cub_call();
    k_invert<<<blocks_for(nn), kThreads, 0, st>>>(bfs2pre, nn, pre2bfs);
    count_launch();
    TPM_CUDA(cudaGetLastError());

    // ---- walk tables and monopoles.  The tables that need no monopole go on
    // the context's side stream while the monopole pass climbs (its last
    // levels leave most SMs idle); the centres of mass follow both.
    NodeOut o{s->ncen, s->ncom,  s->nlink, s->nlevel, s->nprefix, s->bcen,
              s->bcom, s->blink, s->spart, s->nsoft,  s->bsoft};
    TPM_CUDA(cudaEventRecord(c->ev_fork, st));
    TPM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    k_tables<<<blocks_for(nn), kThreads, 0, c->side>>>(t, pre2bfs, nn, spos, smass, s->x0[0], s->x0[1], s->x0[2],
                                                       s->L0, o);
    const cudaError_t e_tab = cudaGetLastError();
    const cudaError_t e_join = cudaEventRecord(c->ev_join, c->side);
    k_multipole<<<blocks_for(nn), kThreads, 0, st>>>(t, nn, pre2bfs, spos, smass, M, S, s->psoft, hmx, hmn);
    const cudaError_t e_mp = cudaGetLastError();
    // st waits for the side stream before anything (the scratch frees among
    // them) follows on it; if that cannot be enqueued, the host waits instead
    const cudaError_t e_wait = e_join == cudaSuccess ? cudaStreamWaitEvent(st, c->ev_join, 0) : e_join;
    if (e_wait != cudaSuccess)
        cudaStreamSynchronize(c->side);
    TPM_CUDA(e_tab);
    TPM_CUDA(e_wait);
    TPM_CUDA(e_mp);
    count_launch(2);
    k_com<<<blocks_for(nn), kThreads, 0, st>>>(t, pre2bfs, nn, M, S, hmx, hmn, s->x0[0], s->x0[1], s->x0[2], s->L0, o);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
