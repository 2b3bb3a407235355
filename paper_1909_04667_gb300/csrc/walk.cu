// Tree walk for the active particles (paper Sec. 3.1, 3.2, 3.4).
//
// One warp walks the tree for a group of 32 active particles that are
// consecutive in key order, hence close in space.  Every lane keeps its own
// particle's opening decisions -- exactly the per-particle walk of the paper
// -- while the warp moves through the depth-first pre-order node array
// together: a node is visited when at least one lane still needs it; a lane
// that accepted a node (or skipped it beyond the short-range cutoff) ignores
// the node's subtree by remembering the subtree's end (the node's skip index)
// and idling until the warp has passed it.  __ballot_sync decides whether the
// warp descends into a node or jumps past it.
//
// Node records are three 16-byte structures (centre + side, centre of mass
// offset + mass, links) read with one vector load each through the read-only
// path; all lanes read the same address, so each load is one broadcast.
//
// Precision: positions are FP64.  Each group works in a frame centred on the
// smallest key cell that holds the whole group; node centres relative to the
// root corner are exact FP32 numbers (they lie on the 2^-22 L0 grid), so the
// node-to-group centre offset is exact in FP32.  Particle positions enter as
// FP64 differences to the group centre, node centres of mass and leaf
// particles as FP32 offsets from their node centre, so every pair vector is
// a sum of small, accurately rounded terms and the pair arithmetic runs in
// FP32 with FP32 accumulation.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kWalkThreads = 256;

struct WalkConsts {
    float h2, hinv, hinv3;
    float thr_const;     // theta^2 (geometric criterion)
    float alpha_over_G;  // relative criterion: open if M L^2 > (alpha |a_old| / G) d^4
    float rcut2, inv2rs;
    float box, boxinv, bigL;
    float G;
    int box_guard;
    int plain;  // 1: the plain FP32 form (absolute FP32 coordinates)
    // Ewald correction (periodic tree without the mesh): unit-box table of
    // (ent + 1)^3 float4, index scale 2 ent / box, force and potential scales
    // 1 / box^2 and 1 / box, and the own-lattice potential at d = 0
    const float4 *etab;
    float escale, efs, eps, ephi0;
    int ent;
};

__device__ __forceinline__ uint32_t compact3w(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x001f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x001f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// Short-range factors of the Gaussian force split (Sec. 3.4) at u = r / 2 r_s:
//   force     g_s = erfc(u) + 2 u / sqrt(pi) exp(-u^2)
//   potential g_p = erfc(u)
// erfc by the rational approximation of Abramowitz & Stegun (1964), eq.
// 7.1.26 (absolute error <= 1.5e-7 for u >= 0), which shares exp(-u^2)
// with the second term.
__device__ __forceinline__ void short_range_factors(float r, float inv2rs, float &gs, float &gp) {
    const float u = r * inv2rs;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, u, 1.0f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    const float e = __expf(-u * u);
    const float erfc_u = poly * e;
    gp = erfc_u;
    gs = fmaf(1.1283791671f * u, e, erfc_u);
}

// Adds the spline-softened (Sec. 3.2) pair term of mass m at offset (rx, ry, rz)
// (source minus target) to the acceleration and potential sums.  With the
// cubic-spline density of support h the force is Newtonian from r = h on.
template <bool TREEPM>
__device__ __forceinline__ void pair_term_s(float rx, float ry, float rz, float r2, float m, float h2, float hinv,
                                            float hinv3, const WalkConsts &k, float &ax, float &ay, float &az,
                                            float &ph) {
    float kf, kp;
    if (r2 >= h2) {
        const float ri = rsqrtf(r2);
        const float ri2 = ri * ri;
        kf = ri * ri2;
        kp = -ri;
        if (TREEPM) {
            float gs, gp;
            short_range_factors(r2 * ri, k.inv2rs, gs, gp);
            kf *= gs;
            kp *= gp;
        }
    } else {
        const float r = sqrtf(r2);
        const float u = r * hinv;
        const float u2 = u * u;
        if (u < 0.5f) {
            kf = hinv3 * fmaf(u2, fmaf(32.0f, u, -38.4f), 10.666666667f);
            kp = hinv * fmaf(u2, fmaf(u2, fmaf(6.4f, u, -9.6f), 5.333333333f), -2.8f);
        } else {
            const float iu = __fdividef(1.0f, u);
            kf = hinv3 * (fmaf(u, fmaf(u, fmaf(-10.666666667f, u, 38.4f), -48.0f), 21.333333333f) -
                            0.066666666667f * iu * iu * iu);
            kp = hinv * (fmaf(u2, fmaf(u, fmaf(u, fmaf(-2.133333333f, u, 9.6f), -16.0f), 10.666666667f), -3.2f) +
                           0.066666666667f * iu);
        }
        if (TREEPM) {
            float gs, gp;
            short_range_factors(r, k.inv2rs, gs, gp);
            kf *= gs;
            kp *= gp;
        }
    }
    const float mk = m * kf;
    ax = fmaf(mk, rx, ax);
    ay = fmaf(mk, ry, ay);
    az = fmaf(mk, rz, az);
    ph = fmaf(m, kp, ph);
}

template <bool TREEPM>
__device__ __forceinline__ void pair_term(float rx, float ry, float rz, float r2, float m, const WalkConsts &k,
                                          float &ax, float &ay, float &az, float &ph) {
    pair_term_s<TREEPM>(rx, ry, rz, r2, m, k.h2, k.hinv, k.hinv3, k, ax, ay, az, ph);
}

// The same pair term with the pair's own spline support h (per-particle
// softening, Sec. 3.2); 1 / h only inside the support.
template <bool TREEPM>
__device__ __forceinline__ void pair_term_h(float rx, float ry, float rz, float r2, float m, float h,
                                            const WalkConsts &k, float &ax, float &ay, float &az, float &ph) {
    const float h2 = h * h;
    float hinv = 0.0f, hinv3 = 0.0f;
    if (r2 < h2) {
        hinv = 1.0f / h;
        hinv3 = hinv * hinv * hinv;
    }
    pair_term_s<TREEPM>(rx, ry, rz, r2, m, h2, hinv, hinv3, k, ax, ay, az, ph);
}


__device__ __forceinline__ float wrap_min_image(float d, const WalkConsts &k) {
    return fmaf(-k.box, rintf(d * k.boxinv), d);
}

// Ewald correction (Sec. 3.1) of mass m at nearest-image offset (rx, ry, rz)
// (source minus target): trilinear interpolation of the table at |r| per
// axis; the force correction is odd in its own component and even in the
// others, the potential correction even in all.
__device__ __forceinline__ void ewald_term(float rx, float ry, float rz, float m, const WalkConsts &k, float &ax,
                                           float &ay, float &az, float &ph) {
    const int top = k.ent - 1, m1 = k.ent + 1;
    const float ux = fabsf(rx) * k.escale, uy = fabsf(ry) * k.escale, uz = fabsf(rz) * k.escale;
    const int ix = min((int)ux, top), iy = min((int)uy, top), iz = min((int)uz, top);
    const float fx = ux - (float)ix, fy = uy - (float)iy, fz = uz - (float)iz;
    const float4 *t = k.etab + ((ix * m1 + iy) * m1 + iz);
    const int sy = m1, sx = m1 * m1;
    const float4 c000 = __ldg(t), c001 = __ldg(t + 1), c010 = __ldg(t + sy), c011 = __ldg(t + sy + 1);
    const float4 c100 = __ldg(t + sx), c101 = __ldg(t + sx + 1), c110 = __ldg(t + sx + sy),
                 c111 = __ldg(t + sx + sy + 1);
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float a00 = (&c000.x)[q] + fz * ((&c001.x)[q] - (&c000.x)[q]);
        const float a01 = (&c010.x)[q] + fz * ((&c011.x)[q] - (&c010.x)[q]);
        const float a10 = (&c100.x)[q] + fz * ((&c101.x)[q] - (&c100.x)[q]);
        const float a11 = (&c110.x)[q] + fz * ((&c111.x)[q] - (&c110.x)[q]);
        const float b0 = a00 + fy * (a01 - a00), b1 = a10 + fy * (a11 - a10);
        v[q] = b0 + fx * (b1 - b0);
    }
    const float mf = m * k.efs;
    ax = fmaf(mf, rx < 0.0f ? -v[0] : v[0], ax);
    ay = fmaf(mf, ry < 0.0f ? -v[1] : v[1], ay);
    az = fmaf(mf, rz < 0.0f ? -v[2] : v[2], az);
    ph = fmaf(m * k.eps, v[3], ph);
}

// Compensated (Kahan) addition s += t with the lost low part kept in c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float t) {
    const float y = t - c;
    const float u = s + y;
    c = (u - s) - y;
    s = u;
}

// One interaction of the periodic tree with the Ewald correction: the pair
// term and its correction are added up first, then into the sums with
// compensation (c), since a particle of a near-uniform box sums some 10^4
// such terms to a small total.
__device__ __forceinline__ void ewald_pair_term(float rx, float ry, float rz, float r2, float m, const WalkConsts &k,
                                                float &ax, float &ay, float &az, float &ph, float4 &c) {
    float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
    pair_term<false>(rx, ry, rz, r2, m, k, tx, ty, tz, tp);
    ewald_term(rx, ry, rz, m, k, tx, ty, tz, tp);
    kahan_add(ax, c.x, tx);
    kahan_add(ay, c.y, ty);
    kahan_add(az, c.z, tz);
    kahan_add(ph, c.w, tp);
}

// ----------------------------------------------------------------------
// Walk frames of spread-out chunks.
//
// A group's frame is the smallest key cell holding its first and last
// particle, and each particle's offset from the frame centre is rounded to
// FP32 once (an error up to 2^-25 of the cell's side).  Particles that are
// consecutive in key order are normally close, but a chunk can reach from a
// dense region to a far particle (an outlier, or a jump of the space-filling
// curve across a coarse cell boundary); its frame is then far coarser than
// the separations of its dense members and their close pairs lose precision.
// Such a chunk is cut into runs: wherever the frame is more than
// 2^kFrameSpan times coarser than the finest cell some member shares with a
// key-order neighbour, the chunk splits at the pairs of consecutive
// particles that share only the frame's cell, and the pieces are examined
// again.  The warp then walks the runs one after the other, each in its own
// frame (the lane walk lists them for a small group-walk launch after it);
// every decision stays the per-particle walk's.
constexpr int kFrameSpan = 8;

__device__ __forceinline__ int common_level(uint64_t a, uint64_t b) {
    const uint64_t x = a ^ b;
    return x ? min((__clzll(x) - 1) / 3, kMaxLevel) : kMaxLevel;
}

// Bit i of the result: a run ends after particle i of the chunk [g0, g0 +
// gcount) of the sorted active list (0: the chunk keeps one frame).
__device__ __forceinline__ unsigned chunk_cuts(const uint64_t *__restrict__ key, const uint32_t *__restrict__ sidx,
                                               int64_t g0, int gcount) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool valid = lane < gcount;
    const int64_t gi = valid ? g0 + lane : g0;
    const uint64_t kk = key[sidx ? sidx[gi] : (uint32_t)gi];
    const uint64_t kn = __shfl_down_sync(FULL, kk, 1);
    const bool pair = lane + 1 < gcount;  // (lane, lane + 1) are consecutive members
    const int lv = pair ? common_level(kk, kn) : 0;
    unsigned cut = 0u;
    for (int it = 0; it <= kMaxLevel; it++) {
        const bool inrun = pair && !((cut >> lane) & 1u);
        const int prev = __shfl_up_sync(FULL, inrun ? lv : -1, 1);
        // finest level this particle shares with an in-run neighbour, and
        // the run's frame level (the coarsest level shared inside the run)
        const int lam = max(inrun ? lv : -1, lane > 0 ? prev : -1);
        const unsigned run = valid ? (unsigned)__popc(cut & ((1u << lane) - 1u)) : 64u + (unsigned)lane;
        const unsigned seg = __match_any_sync(FULL, run);
        const unsigned frame = __reduce_min_sync(seg, inrun ? (unsigned)lv : 99u);
        const unsigned finest = __reduce_max_sync(seg, (unsigned)(lam + 1));
        const bool split = valid && inrun && (unsigned)lv == frame && finest > frame + 1u + (unsigned)kFrameSpan;
        const unsigned add = __ballot_sync(FULL, split);
        if (!add)
            break;
        cut |= add;
    }
    return cut;
}

// Appends the runs of a cut chunk to the run list (start, count).
__device__ __forceinline__ void append_runs(unsigned cut, int64_t g0, int gcount, uint2 *__restrict__ runs,
                                            unsigned *__restrict__ nruns) {
    const int lane = threadIdx.x & 31;
    const unsigned starts = (1u | (cut << 1)) & (gcount >= 32 ? 0xffffffffu : ((1u << gcount) - 1u));
    unsigned base = 0;
    if (lane == 0)
        base = atomicAdd(nruns, (unsigned)__popc(starts));
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((starts >> lane) & 1u) {
        const unsigned long long above = (unsigned long long)starts & ~((2ull << lane) - 1ull);
        const int next = above ? __ffsll((long long)above) - 1 : gcount;
        runs[base + __popc(starts & ((1u << lane) - 1u))] = make_uint2((uint32_t)(g0 + lane), (uint32_t)(next - lane));
    }
}

template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk(const float4 *__restrict__ ncen, const float4 *__restrict__ ncom, const int4 *__restrict__ nlink,
           const float4 *__restrict__ spart, const uint64_t *__restrict__ key, const uint32_t *__restrict__ perm,
           const double *__restrict__ pos, double x0, double y0, double z0, double L0, int nnodes,
           const float *__restrict__ psoft, const float *__restrict__ nsoft, const uint32_t *__restrict__ sidx,
           const uint32_t *__restrict__ slot, const float *__restrict__ a_old, int64_t n_act, WalkConsts k,
           float *__restrict__ acc, float *__restrict__ pot, uint32_t *__restrict__ nint, int accumulate,
           uint2 *__restrict__ runs, unsigned *__restrict__ nruns) {
    constexpr bool EWALD = PERIODIC && !TREEPM;  // periodic tree without the mesh
    const int lane = threadIdx.x & 31;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane);
    if (g0 >= n_act)
        return;  // the whole warp leaves together
    if (!PERIODIC && !k.plain) {  // spread-out chunks are walked in runs by the group walk
        const int gcount = (int)min((int64_t)32, n_act - g0);
        const unsigned cut = chunk_cuts(key, sidx, g0, gcount);
        if (cut) {
            append_runs(cut, g0, gcount, runs, nruns);
            return;
        }
    }
    const int64_t gi = g0 + lane;
    const bool valid = gi < n_act;
    const int64_t glast = min(g0 + 31, n_act - 1);
    const uint32_t s = sidx ? sidx[valid ? gi : g0] : (uint32_t)(valid ? gi : g0);
    const uint32_t s_first = sidx ? sidx[g0] : (uint32_t)g0;
    const uint32_t s_last = sidx ? sidx[glast] : (uint32_t)glast;
    const uint32_t out = slot ? slot[valid ? gi : g0] : perm[s];

    // group frame: the smallest key cell holding the group's first and last particle
    const uint64_t kf = key[s_first], kl = key[s_last];
    const uint64_t kx = kf ^ kl;
    const int glevel = kx ? min((__clzll(kx) - 1) / 3, kMaxLevel) : kMaxLevel;
    const uint64_t gpre = kf >> (3 * (kMaxLevel - glevel));
    const double ghalf = ldexp(L0, -(glevel + 1));
    const bool abs_frame = !PERIODIC && k.plain;  // the plain FP32 form: absolute FP32 coordinates
    const double gcx_d = abs_frame ? -x0 : (double)(2 * (uint64_t)compact3w(gpre) + 1) * ghalf;
    const double gcy_d = abs_frame ? -y0 : (double)(2 * (uint64_t)compact3w(gpre >> 1) + 1) * ghalf;
    const double gcz_d = abs_frame ? -z0 : (double)(2 * (uint64_t)compact3w(gpre >> 2) + 1) * ghalf;
    const float gcx = (float)gcx_d, gcy = (float)gcy_d, gcz = (float)gcz_d;
    const uint32_t j = perm[s];
    const float xox = (float)(pos[3 * j] - (x0 + gcx_d));
    const float xoy = (float)(pos[3 * j + 1] - (y0 + gcy_d));
    const float xoz = (float)(pos[3 * j + 2] - (z0 + gcz_d));

    float thr = k.thr_const;
    if (RELATIVE)
        thr = valid ? k.alpha_over_G * fabsf(a_old[out]) : 0.0f;
    const float hi = VARH ? __ldg(&psoft[s]) : 0.0f;  // this particle's spline support

    float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
    float4 ec = make_float4(0.f, 0.f, 0.f, 0.f);  // compensation of the Ewald sums
    uint32_t cnt = 0;
    int skip_until = valid ? 0 : 0x7fffffff;
    int n = 0;
    while (n < nnodes) {
        const float4 C = __ldg(&ncen[n]);
        const float4 O = __ldg(&ncom[n]);
        const int4 Lk = __ldg(&nlink[n]);
        const bool act = n >= skip_until;
        const float dcx = C.x - gcx, dcy = C.y - gcy, dcz = C.z - gcz;  // exact
        float px = xox - dcx, py = xoy - dcy, pz = xoz - dcz;  // particle relative to node centre
        if (PERIODIC) {  // nearest image of the node centre as seen from this particle
            px = wrap_min_image(px, k);
            py = wrap_min_image(py, k);
            pz = wrap_min_image(pz, k);
        }
        const float L = C.w;
        float rx = O.x - px, ry = O.y - py, rz = O.z - pz;  // particle -> centre of mass
        if (PERIODIC && (EWALD || L > k.bigL)) {  // the Ewald table needs the nearest image
            rx = wrap_min_image(rx, k);
            ry = wrap_min_image(ry, k);
            rz = wrap_min_image(rz, k);
        }
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        bool far = false;
        if (TREEPM) {
            const float ex = fmaxf(fabsf(px) - 0.5f * L, 0.0f), ey = fmaxf(fabsf(py) - 0.5f * L, 0.0f),
                        ez = fmaxf(fabsf(pz) - 0.5f * L, 0.0f);
            far = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > k.rcut2;
        }
        const float gl = 0.6f * L;
        const bool guard = k.box_guard && fabsf(px) <= gl && fabsf(py) <= gl && fabsf(pz) <= gl;
        bool crit;
        if (RELATIVE)
            crit = O.w * L * L > thr * r2 * r2;
        else
            crit = L * L > thr * r2;
        float hn = 0.0f;
        if (VARH) {  // Sec. 3.2: a node of mixed softenings is opened inside its largest one
            const float v = __ldg(&nsoft[n]);
            hn = fabsf(v);
            crit = crit || (v < 0.0f && hi < hn && r2 < hn * hn);
        }
        const bool open = act && !far && (guard || crit);
        if (act && !open) {
            if (!far) {
                if (EWALD)
                    ewald_pair_term(rx, ry, rz, r2, O.w, k, ax, ay, az, ph, ec);
                else if (VARH)
                    pair_term_h<TREEPM>(rx, ry, rz, r2, O.w, fmaxf(hi, hn), k, ax, ay, az, ph);
                else
                    pair_term<TREEPM>(rx, ry, rz, r2, O.w, k, ax, ay, az, ph);
                cnt++;
            }
            skip_until = Lk.x;
        }
        const unsigned want = __ballot_sync(0xffffffffu, open);
        if (want == 0u) {
            n = Lk.x;
            continue;
        }
        if (!Lk.w) {
            n = n + 1;  // first child follows in pre-order
            continue;
        }
        // opened leaf: particle by particle
        const int jend = Lk.y + Lk.z;
        for (int jj = Lk.y; jj < jend; jj++) {
            const float4 P = __ldg(&spart[jj]);
            if (open && (uint32_t)jj != s) {
                float qx = P.x - px, qy = P.y - py, qz = P.z - pz;
                if (PERIODIC && (EWALD || L > k.bigL)) {
                    qx = wrap_min_image(qx, k);
                    qy = wrap_min_image(qy, k);
                    qz = wrap_min_image(qz, k);
                }
                const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                if (!TREEPM || q2 <= k.rcut2) {
                    if (EWALD)
                        ewald_pair_term(qx, qy, qz, q2, P.w, k, ax, ay, az, ph, ec);
                    else if (VARH)
                        pair_term_h<TREEPM>(qx, qy, qz, q2, P.w, fmaxf(hi, __ldg(&psoft[jj])), k, ax, ay, az, ph);
                    else
                        pair_term<TREEPM>(qx, qy, qz, q2, P.w, k, ax, ay, az, ph);
                    cnt++;
                }
            }
        }
        n = Lk.x;
    }
    if (!valid)
        return;
    if (EWALD)  // the particle's own images and the background
        ph = fmaf(__ldg(&spart[s]).w * k.eps, k.ephi0, ph);
    const float G = k.G;
    if (accumulate) {
        acc[3 * (size_t)out] += G * ax;
        acc[3 * (size_t)out + 1] += G * ay;
        acc[3 * (size_t)out + 2] += G * az;
        if (pot)
            pot[out] += G * ph;
    } else {
        acc[3 * (size_t)out] = G * ax;
        acc[3 * (size_t)out + 1] = G * ay;
        acc[3 * (size_t)out + 2] = G * az;
        if (pot)
            pot[out] = G * ph;
    }
    if (nint)
        nint[out] = cnt;
}

// ======================================================================
// Group walk.
//
// The lane walk above pays ~50 warp instructions for every node it visits,
// however few lanes need the node.  Most visited nodes, though, get the same
// answer from every particle of a compact group: far nodes are accepted by
// all, nearby ones opened by all, and with TreePM distant ones skipped by all.
// The group walk therefore decides each candidate node once for the whole
// group, one node per lane, from the group's bounding box with conservative
// bounds (a node is "accepted by all" only if the criterion accepts it even
// for the box point closest to its centre of mass, and so on), and keeps the
// per-particle decision only for the nodes where the bounds leave doubt:
// those are resolved lane by lane exactly as in the lane walk, and a lane that
// accepts such a node adds its monopole right away.  The decisions
// -- hence every particle's interaction set -- are the per-particle walk's.
// Accepted nodes and opened leaves go to a per-warp list in shared memory,
// tagged with the lanes they apply to, and the lanes then sweep the list in a
// tight loop of pair terms.  Candidates come from a per-warp stack of child
// ranges (children are contiguous in breadth-first order).
// ======================================================================
constexpr int kGroupWarps = 4;
// Candidate-stack capacity: 192 for the plain walk; the batched walk is also
// compiled at 128 and 256 for the plan's autotuner.  Above capacity - 64
// entries the walk takes one candidate at a time, so the stack grows by at
// most one batch of pushes (32) plus the tree depth (21) past that mark.
constexpr int kStackCap = 192;
constexpr int kStackDepths[3] = {128, 192, 256};
constexpr int kNodeFlush = 64;              // sweep once this many node entries are queued
constexpr int kNodeCap = kNodeFlush + 32;   // one step adds at most 32 (one per lane)
constexpr int kLeafFlush = 32;
constexpr int kLeafCap = kLeafFlush + 32;
constexpr int kUndCap = 96;                 // nodes waiting for per-particle decisions
constexpr uint32_t kLeafWrap = 0x80000000u, kLeafCount = 0x7fffffffu;
enum { kSkip = 0, kAccept = 1, kOpen = 2, kMixed = 3, kNone = 4 };

template <int STACK, bool VARH, bool PERIODIC>
struct GroupSharedT {
    static constexpr int kStack = STACK;
    static constexpr int kSafe = STACK - 64;  // above this, take one candidate at a time
    uint2 stack[STACK];  // (first child, lane mask)
    uint8_t scount[STACK];
    // accepted node e: centre of mass (group frame) and mass, stored by pairs
    // of entries so that one 128-bit load feeds the two-wide FP32
    // instructions: nxy[e / 2] = (x, x', y, y'), nzm[e / 2] = (z, z', m, m')
    float4 nxy[kNodeCap / 2];
    float4 nzm[kNodeCap / 2];
    uint32_t nmask[kNodeCap];
    float nsoft[VARH ? kNodeCap : 1];      // its largest spline support (per-particle softening)
    uint8_t nwrap[PERIODIC ? kNodeCap : 1];
    float4 lsrc[kLeafCap];   // opened leaf: centre (group frame) + first particle
    uint2 lmeta[kLeafCap];   // lane mask, wrap flag | particle count
    uint2 und[kUndCap];      // node the group bounds left undecided, lane mask
    // the group's particles by pairs: offset from the frame centre and
    // criterion threshold, pxy[i] = (x, x', y, y'), pzt[i] = (z, z', t, t')
    float4 pxy[16];
    float4 pzt[16];
};

// Entry e of the node queue (paired layout).
template <class SH>
__device__ __forceinline__ float4 node_entry(const SH &sh, int e) {
    const float *a = reinterpret_cast<const float *>(&sh.nxy[e >> 1]);
    const float *b = reinterpret_cast<const float *>(&sh.nzm[e >> 1]);
    const int o = e & 1;
    return make_float4(a[o], a[2 + o], b[o], b[2 + o]);
}

template <class SH>
__device__ __forceinline__ void put_node_entry(SH &sh, int e, float4 v) {
    float *a = reinterpret_cast<float *>(&sh.nxy[e >> 1]);
    float *b = reinterpret_cast<float *>(&sh.nzm[e >> 1]);
    const int o = e & 1;
    a[o] = v.x;
    a[2 + o] = v.y;
    b[o] = v.z;
    b[2 + o] = v.w;
}

template <class SH>
__device__ __forceinline__ void put_part_entry(SH &sh, int p, float4 v) {
    float *a = reinterpret_cast<float *>(&sh.pxy[p >> 1]);
    float *b = reinterpret_cast<float *>(&sh.pzt[p >> 1]);
    const int o = p & 1;
    a[o] = v.x;
    a[2 + o] = v.y;
    b[o] = v.z;
    b[2 + o] = v.w;
}

// Particle p of the group (paired layout): offset and criterion threshold.
template <class SH>
__device__ __forceinline__ float4 part_entry(const SH &sh, int p) {
    const float *a = reinterpret_cast<const float *>(&sh.pxy[p >> 1]);
    const float *b = reinterpret_cast<const float *>(&sh.pzt[p >> 1]);
    const int o = p & 1;
    return make_float4(a[o], a[2 + o], b[o], b[2 + o]);
}

// Conservative decision for all particles inside [lo, hi] (group frame).
template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH>
__device__ __forceinline__ int classify_group(float4 C, float4 O, float gcx, float gcy, float gcz, float lox,
                                              float loy, float loz, float hix, float hiy, float hiz, float thr_min,
                                              float thr_max, bool wide, float hsig, float hmin_g, const WalkConsts &k,
                                              float &dcx, float &dcy, float &dcz) {
    dcx = C.x - gcx;
    dcy = C.y - gcy;
    dcz = C.z - gcz;
    if (PERIODIC) {
        dcx = wrap_min_image(dcx, k);
        dcy = wrap_min_image(dcy, k);
        dcz = wrap_min_image(dcz, k);
    }
    const float L = C.w, M = O.w;
    if (PERIODIC && (wide || L > k.bigL))
        return kMixed;  // the group-centred image may not be every particle's nearest one
    const float up = 1.0f + 1e-5f, dn = 1.0f - 1e-5f;
    // range of (particle - node centre) over the box, per axis
    const float ax0 = lox - dcx, ax1 = hix - dcx, ay0 = loy - dcy, ay1 = hiy - dcy, az0 = loz - dcz, az1 = hiz - dcz;
    const float nx = fmaxf(fmaxf(ax0, -ax1), 0.0f), ny = fmaxf(fmaxf(ay0, -ay1), 0.0f),
                nz = fmaxf(fmaxf(az0, -az1), 0.0f);  // nearest |p - c|
    const float fx = fmaxf(fabsf(ax0), fabsf(ax1)), fy = fmaxf(fabsf(ay0), fabsf(ay1)),
                fz = fmaxf(fabsf(az0), fabsf(az1));  // farthest |p - c|
    bool maybe_far = false;  // some particles may see the node beyond the cutoff
    if (TREEPM) {
        const float hL = 0.5f * L;
        const float ex = fmaxf(nx - hL, 0.0f), ey = fmaxf(ny - hL, 0.0f), ez = fmaxf(nz - hL, 0.0f);
        if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > k.rcut2 * up)
            return kSkip;
        const float gx = fmaxf(fx - hL, 0.0f), gy = fmaxf(fy - hL, 0.0f), gz = fmaxf(fz - hL, 0.0f);
        maybe_far = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > k.rcut2 * dn;
    }
    const float gl = 0.6f * L;
    const bool guard_all = k.box_guard && fmaxf(fx, fmaxf(fy, fz)) <= gl * dn;
    const bool guard_none = !k.box_guard || fmaxf(nx, fmaxf(ny, nz)) > gl * up;
    // range of (particle - centre of mass)
    const float cx = dcx + O.x, cy = dcy + O.y, cz = dcz + O.z;
    const float bx0 = lox - cx, bx1 = hix - cx, by0 = loy - cy, by1 = hiy - cy, bz0 = loz - cz, bz1 = hiz - cz;
    const float mx = fmaxf(fmaxf(bx0, -bx1), 0.0f), my = fmaxf(fmaxf(by0, -by1), 0.0f),
                mz = fmaxf(fmaxf(bz0, -bz1), 0.0f);
    const float Mx = fmaxf(fabsf(bx0), fabsf(bx1)), My = fmaxf(fabsf(by0), fabsf(by1)),
                Mz = fmaxf(fabsf(bz0), fabsf(bz1));
    // without the cutoff (Ewald tree) nodes near half a box away occur: when a
    // particle of the group may see another image of the centre or the
    // centre of mass than the group-centred one, decide per particle
    if (PERIODIC && !TREEPM && fmaxf(fmaxf(fmaxf(fx, fy), fz), fmaxf(fmaxf(Mx, My), Mz)) >= 0.5f * k.box * dn)
        return kMixed;
    const float dmin2 = fmaf(mx, mx, fmaf(my, my, mz * mz));
    const float dmax2 = fmaf(Mx, Mx, fmaf(My, My, Mz * Mz));
    bool open_all, acc_all;
    if (RELATIVE) {
        const float q = M * L * L;
        open_all = q > thr_max * dmax2 * dmax2 * up;
        acc_all = q <= thr_min * dmin2 * dmin2 * dn;
    } else {
        const float q = L * L;
        open_all = q > k.thr_const * dmax2 * up;
        acc_all = q <= k.thr_const * dmin2 * dn;
    }
    if (VARH && hsig < 0.0f && hmin_g < -hsig && dmin2 < hsig * hsig)
        acc_all = false;  // Sec. 3.2: some particle may have to open this node of mixed softenings
    // Opening for all is exact even when the node lies beyond the cutoff for
    // some particles: for them every descendant does too, and the leaf sweep
    // drops pairs beyond the cutoff, so they gain no interaction.  Accepting
    // needs every particle inside the cutoff.
    if (guard_all || open_all)
        return kOpen;
    if (!maybe_far && guard_none && acc_all)
        return kAccept;
    return kMixed;
}

// Monopole of mass m at offset (rx, ry, rz) for r2 >= h2 (Newtonian, no split).
__device__ __forceinline__ void newton_term(float rx, float ry, float rz, float r2, float m, float &ax, float &ay,
                                            float &az, float &ph) {
    const float ri = rsqrtf(r2);
    const float mr = m * ri;
    const float mr3 = mr * ri * ri;
    ax = fmaf(mr3, rx, ax);
    ay = fmaf(mr3, ry, ay);
    az = fmaf(mr3, rz, az);
    ph -= mr;
}

// Node entries accepted by every particle of the group sit at the front of the
// node queue: no lane masks, straight-line Newtonian terms four at a time.
// With one softening length h every entry first gets the Newtonian term at
// max(r, h); when some lane met an entry closer than h (its smallest r^2 is
// below h^2, rare for accepted nodes), a second pass takes the h-term of those
// entries out again and adds their spline term.  With per-particle softening
// (VARH) the support of an entry is the larger of the lane's own (hi) and the
// node's largest (Sec. 3.2), and such entries add zero mass in the first pass.
template <bool PERIODIC, bool TREEPM, bool VARH, class SH>
__device__ __forceinline__ void sweep_full(const SH &sh, int nf, float xox, float xoy, float xoz, float hi,
                                           const WalkConsts &k, float &ax, float &ay, float &az, float &ph,
                                           float4 &ec) {
    if (TREEPM || PERIODIC) {
        for (int e = 0; e < nf; e++) {
            const float4 A = node_entry(sh, e);
            float rx = A.x - xox, ry = A.y - xoy, rz = A.z - xoz;
            if (PERIODIC && sh.nwrap[e]) {
                rx = wrap_min_image(rx, k);
                ry = wrap_min_image(ry, k);
                rz = wrap_min_image(rz, k);
            }
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            if (PERIODIC && !TREEPM)
                ewald_pair_term(rx, ry, rz, r2, A.w, k, ax, ay, az, ph, ec);
            else if (VARH)
                pair_term_h<TREEPM>(rx, ry, rz, r2, A.w, fmaxf(hi, sh.nsoft[e]), k, ax, ay, az, ph);
            else
                pair_term<TREEPM>(rx, ry, rz, r2, A.w, k, ax, ay, az, ph);
        }
        return;
    }
    if (!VARH) {
        // pairs of entries through the two-wide FP32 instructions, each
        // element rounded as the scalar instruction would round it; the two
        // halves of each sum are added at the end
        float rmin = __int_as_float(0x7f800000);
        const float2 nx = make_float2(-xox, -xox), ny = make_float2(-xoy, -xoy), nz = make_float2(-xoz, -xoz);
        float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx, sp = sx;
        int e = 0;
#pragma unroll 2
        for (; e + 1 < nf; e += 2) {
            const float4 XY = sh.nxy[e >> 1], ZM = sh.nzm[e >> 1];
            const float2 rx = __fadd2_rn(make_float2(XY.x, XY.y), nx);
            const float2 ry = __fadd2_rn(make_float2(XY.z, XY.w), ny);
            const float2 rz = __fadd2_rn(make_float2(ZM.x, ZM.y), nz);
            const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
            rmin = fminf(rmin, fminf(r2.x, r2.y));
            const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, k.h2)), rsqrtf(fmaxf(r2.y, k.h2)));
            const float2 mr = __fmul2_rn(make_float2(ZM.z, ZM.w), ri);
            const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
            sx = __ffma2_rn(mr3, rx, sx);
            sy = __ffma2_rn(mr3, ry, sy);
            sz = __ffma2_rn(mr3, rz, sz);
            sp = __fadd2_rn(sp, mr);
        }
        ax += sx.x + sx.y;
        ay += sy.x + sy.y;
        az += sz.x + sz.y;
        ph -= sp.x + sp.y;
        for (; e < nf; e++) {
            const float4 A = node_entry(sh, e);
            const float rx = A.x - xox, ry = A.y - xoy, rz = A.z - xoz;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            rmin = fminf(rmin, r2);
            newton_term(rx, ry, rz, fmaxf(r2, k.h2), A.w, ax, ay, az, ph);
        }
        if (__any_sync(0xffffffffu, rmin < k.h2)) {
            for (int q = 0; q < nf; q++) {
                const float4 A = node_entry(sh, q);
                const float rx = A.x - xox, ry = A.y - xoy, rz = A.z - xoz;
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                if (r2 < k.h2) {
                    newton_term(rx, ry, rz, k.h2, -A.w, ax, ay, az, ph);
                    pair_term<false>(rx, ry, rz, r2, A.w, k, ax, ay, az, ph);
                }
            }
        }
        return;
    }
    bool soft = false;
    int e = 0;
    for (; e + 3 < nf; e += 4) {
        float4 A[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            A[u] = node_entry(sh, e + u);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float rx = A[u].x - xox, ry = A[u].y - xoy, rz = A[u].z - xoz;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            float h2 = k.h2;
            if (VARH) {
                const float he = fmaxf(hi, sh.nsoft[e + u]);
                h2 = he * he;
            }
            const bool sf = r2 < h2;
            soft |= sf;
            newton_term(rx, ry, rz, sf ? h2 : r2, sf ? 0.0f : A[u].w, ax, ay, az, ph);
        }
    }
    for (; e < nf; e++) {
        const float4 A = node_entry(sh, e);
        const float rx = A.x - xox, ry = A.y - xoy, rz = A.z - xoz;
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        float h2 = k.h2;
        if (VARH) {
            const float he = fmaxf(hi, sh.nsoft[e]);
            h2 = he * he;
        }
        const bool sf = r2 < h2;
        soft |= sf;
        newton_term(rx, ry, rz, sf ? h2 : r2, sf ? 0.0f : A.w, ax, ay, az, ph);
    }
    if (__any_sync(0xffffffffu, soft)) {
        for (int q = 0; q < nf; q++) {
            const float4 A = node_entry(sh, q);
            const float rx = A.x - xox, ry = A.y - xoy, rz = A.z - xoz;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            if (VARH) {
                const float he = fmaxf(hi, sh.nsoft[q]);
                if (r2 < he * he)
                    pair_term_h<false>(rx, ry, rz, r2, A.w, he, k, ax, ay, az, ph);
            } else if (r2 < k.h2) {
                pair_term<false>(rx, ry, rz, r2, A.w, k, ax, ay, az, ph);
            }
        }
    }
}

// Node entries for a subset of the lanes sit at the back of the node queue
// (indices [kNodeCap - np, kNodeCap)): a lane not tagged adds a zero mass
// (at max(r, h), since such a lane may sit on the node), and entries inside
// the softening length are repaired as in sweep_full.
template <bool PERIODIC, bool TREEPM, bool VARH, class SH>
__device__ __forceinline__ void sweep_partial(const SH &sh, int np, unsigned lanebit, float xox, float xoy,
                                              float xoz, float hi, const WalkConsts &k, float &ax, float &ay,
                                              float &az, float &ph, uint32_t &cnt, float4 &ec) {
    const int e0 = kNodeCap - np;
    if (TREEPM || PERIODIC) {
        for (int e = e0; e < kNodeCap; e++) {
            const float4 E = node_entry(sh, e);
            const bool mine = (sh.nmask[e] & lanebit) != 0u;
            float rx = E.x - xox, ry = E.y - xoy, rz = E.z - xoz;
            if (PERIODIC && sh.nwrap[e]) {
                rx = wrap_min_image(rx, k);
                ry = wrap_min_image(ry, k);
                rz = wrap_min_image(rz, k);
            }
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            cnt += mine ? 1u : 0u;
            if (PERIODIC && !TREEPM)
                ewald_pair_term(rx, ry, rz, mine ? r2 : 1.0f, mine ? E.w : 0.0f, k, ax, ay, az, ph, ec);
            else if (VARH)
                pair_term_h<TREEPM>(rx, ry, rz, mine ? r2 : 1.0f, mine ? E.w : 0.0f, fmaxf(hi, sh.nsoft[e]), k, ax,
                                    ay, az, ph);
            else
                pair_term<TREEPM>(rx, ry, rz, mine ? r2 : 1.0f, mine ? E.w : 0.0f, k, ax, ay, az, ph);
        }
        return;
    }
    if (!VARH) {
        float rmin = __int_as_float(0x7f800000);
        int e = e0;
        if (e & 1) {  // an odd first entry, then aligned pairs (kNodeCap is even)
            const float4 E = node_entry(sh, e);
            const bool mine = (sh.nmask[e] & lanebit) != 0u;
            const float rx = E.x - xox, ry = E.y - xoy, rz = E.z - xoz;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            rmin = fminf(rmin, r2);
            cnt += mine ? 1u : 0u;
            newton_term(rx, ry, rz, fmaxf(r2, k.h2), mine ? E.w : 0.0f, ax, ay, az, ph);
            e++;
        }
        const float2 nx = make_float2(-xox, -xox), ny = make_float2(-xoy, -xoy), nz = make_float2(-xoz, -xoz);
        float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx, sp = sx;
#pragma unroll 2
        for (; e < kNodeCap; e += 2) {
            const float4 XY = sh.nxy[e >> 1], ZM = sh.nzm[e >> 1];
            const uint2 Mk = *reinterpret_cast<const uint2 *>(&sh.nmask[e]);
            const bool m0 = (Mk.x & lanebit) != 0u, m1 = (Mk.y & lanebit) != 0u;
            const float2 rx = __fadd2_rn(make_float2(XY.x, XY.y), nx);
            const float2 ry = __fadd2_rn(make_float2(XY.z, XY.w), ny);
            const float2 rz = __fadd2_rn(make_float2(ZM.x, ZM.y), nz);
            const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
            rmin = fminf(rmin, fminf(r2.x, r2.y));
            cnt += (m0 ? 1u : 0u) + (m1 ? 1u : 0u);
            const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, k.h2)), rsqrtf(fmaxf(r2.y, k.h2)));
            const float2 mr = __fmul2_rn(make_float2(m0 ? ZM.z : 0.0f, m1 ? ZM.w : 0.0f), ri);
            const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
            sx = __ffma2_rn(mr3, rx, sx);
            sy = __ffma2_rn(mr3, ry, sy);
            sz = __ffma2_rn(mr3, rz, sz);
            sp = __fadd2_rn(sp, mr);
        }
        ax += sx.x + sx.y;
        ay += sy.x + sy.y;
        az += sz.x + sz.y;
        ph -= sp.x + sp.y;
        if (__any_sync(0xffffffffu, rmin < k.h2)) {
            for (int e = e0; e < kNodeCap; e++) {
                const float4 E = node_entry(sh, e);
                const float rx = E.x - xox, ry = E.y - xoy, rz = E.z - xoz;
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                if ((sh.nmask[e] & lanebit) && r2 < k.h2) {
                    newton_term(rx, ry, rz, k.h2, -E.w, ax, ay, az, ph);
                    pair_term<false>(rx, ry, rz, r2, E.w, k, ax, ay, az, ph);
                }
            }
        }
        return;
    }
    bool soft = false;
#pragma unroll 2
    for (int e = e0; e < kNodeCap; e++) {
        const float4 E = node_entry(sh, e);
        const bool mine = (sh.nmask[e] & lanebit) != 0u;
        const float rx = E.x - xox, ry = E.y - xoy, rz = E.z - xoz;
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        float h2 = k.h2;
        if (VARH) {
            const float he = fmaxf(hi, sh.nsoft[e]);
            h2 = he * he;
        }
        const bool sf = r2 < h2;
        soft |= mine && sf;
        const bool use = mine && !sf;
        cnt += mine ? 1u : 0u;
        newton_term(rx, ry, rz, use ? r2 : h2, use ? E.w : 0.0f, ax, ay, az, ph);
    }
    if (__any_sync(0xffffffffu, soft)) {
        for (int e = e0; e < kNodeCap; e++) {
            const float4 E = node_entry(sh, e);
            const float rx = E.x - xox, ry = E.y - xoy, rz = E.z - xoz;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            if (!(sh.nmask[e] & lanebit))
                continue;
            if (VARH) {
                const float he = fmaxf(hi, sh.nsoft[e]);
                if (r2 < he * he)
                    pair_term_h<false>(rx, ry, rz, r2, E.w, he, k, ax, ay, az, ph);
            } else if (r2 < k.h2) {
                pair_term<false>(rx, ry, rz, r2, E.w, k, ax, ay, az, ph);
            }
        }
    }
}

// Sweeps the queued opened leaves, particle by particle.  With open
// boundaries and no split every pair first gets the Newtonian term at
// max(r, h) (no branch: the pairs of a leaf are mostly for a few lanes, and
// many lie inside the softening length); a leaf in which some lane met a
// particle closer than its softening length is swept a second time, taking
// those pairs' h-terms out again and adding their spline terms.
template <bool PERIODIC, bool TREEPM, bool VARH, class SH>
__device__ __forceinline__ void sweep_leaves(const SH &sh, int nl, unsigned lanebit, uint32_t self,
                                             float xox, float xoy, float xoz, float hi,
                                             const float4 *__restrict__ spart, const float *__restrict__ psoft,
                                             const WalkConsts &k, float &ax, float &ay, float &az, float &ph,
                                             uint32_t &cnt, float4 &ec) {
    if (!TREEPM && !PERIODIC) {
        for (int e = 0; e < nl; e++) {
            const float4 E = sh.lsrc[e];
            const uint2 Mt = sh.lmeta[e];
            const bool mine = (Mt.x & lanebit) != 0u;
            // subtract the small particle-to-leaf-centre vector first so that
            // close pairs keep their precision
            const float px = xox - E.x, py = xoy - E.y, pz = xoz - E.z;
            const int j0 = __float_as_int(E.w);
            const int j1 = j0 + (int)(Mt.y & kLeafCount);
            bool close = false;
            for (int jj = j0; jj < j1; jj++) {
                const float4 P = __ldg(&spart[jj]);
                const float qx = P.x - px, qy = P.y - py, qz = P.z - pz;
                const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                float h2 = k.h2;
                if (VARH) {
                    const float he = fmaxf(hi, __ldg(&psoft[jj]));
                    h2 = he * he;
                }
                const bool use = mine && (uint32_t)jj != self;
                close |= use && q2 < h2;
                cnt += use ? 1u : 0u;
                newton_term(qx, qy, qz, fmaxf(q2, h2), use ? P.w : 0.0f, ax, ay, az, ph);
            }
            if (__any_sync(0xffffffffu, close)) {
                for (int jj = j0; jj < j1; jj++) {
                    const float4 P = __ldg(&spart[jj]);
                    const float qx = P.x - px, qy = P.y - py, qz = P.z - pz;
                    const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                    float he = 0.0f, h2 = k.h2;
                    if (VARH) {
                        he = fmaxf(hi, __ldg(&psoft[jj]));
                        h2 = he * he;
                    }
                    if (mine && (uint32_t)jj != self && q2 < h2) {
                        newton_term(qx, qy, qz, h2, -P.w, ax, ay, az, ph);
                        if (VARH)
                            pair_term_h<false>(qx, qy, qz, q2, P.w, he, k, ax, ay, az, ph);
                        else
                            pair_term<false>(qx, qy, qz, q2, P.w, k, ax, ay, az, ph);
                    }
                }
            }
        }
        return;
    }
    for (int e = 0; e < nl; e++) {
        const float4 E = sh.lsrc[e];
        const uint2 Mt = sh.lmeta[e];
        const bool mine = (Mt.x & lanebit) != 0u;
        const bool wr = PERIODIC && (Mt.y & kLeafWrap);
        // subtract the small particle-to-leaf-centre vector first so that close
        // pairs keep their precision
        float px = xox - E.x, py = xoy - E.y, pz = xoz - E.z;
        if (wr) {
            px = wrap_min_image(px, k);
            py = wrap_min_image(py, k);
            pz = wrap_min_image(pz, k);
        }
        const int j0 = __float_as_int(E.w);
        const int j1 = j0 + (int)(Mt.y & kLeafCount);
        for (int jj = j0; jj < j1; jj++) {
            const float4 P = __ldg(&spart[jj]);
            float qx = P.x - px, qy = P.y - py, qz = P.z - pz;
            if (wr) {
                qx = wrap_min_image(qx, k);
                qy = wrap_min_image(qy, k);
                qz = wrap_min_image(qz, k);
            }
            const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
            if (mine && (uint32_t)jj != self && (!TREEPM || q2 <= k.rcut2)) {
                if (PERIODIC && !TREEPM)
                    ewald_pair_term(qx, qy, qz, q2, P.w, k, ax, ay, az, ph, ec);
                else if (VARH)
                    pair_term_h<TREEPM>(qx, qy, qz, q2, P.w, fmaxf(hi, __ldg(&psoft[jj])), k, ax, ay, az, ph);
                else
                    pair_term<TREEPM>(qx, qy, qz, q2, P.w, k, ax, ay, az, ph);
                cnt++;
            }
        }
    }
}

// A tree as the group walk sees it (breadth-first node records, leaf
// particles, keys and positions).
struct TreeView {
    const float4 *bcen, *bcom;
    const int4 *blink;
    const float4 *spart;
    const float *psoft, *bsoft;  // per-particle softening, else null
    const uint64_t *key;
    const uint32_t *perm;
    const double *pos;
    double x0, y0, z0, L0;
};

// Walks the tree for the group of gcount <= 32 active particles at positions
// [g0, g0 + gcount) of the sorted active list (one per lane).
//
// Candidates come from the stack 32 at a time and are classified one per
// lane with the group bounds.  Nodes the bounds leave undecided wait in a
// queue; once 32 wait (or the stack runs dry) they are decided particle by
// particle with the loop transposed: each lane holds one waiting node and
// runs through the group's particles (read from shared memory), so that one
// pass of 32 iterations decides 32 nodes for all 32 particles.  Each
// particle's decision is the per-particle walk's (the same FP32 arithmetic
// as the lane walk); lanes that accept a node get its monopole through the
// node queue, lanes that open it get its children or its leaf.
template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH, class SH>
__device__ __forceinline__ void group_walk(const TreeView &T, const WalkConsts &k, SH &sh,
                                           const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                                           int64_t g0, int gcount, const float *__restrict__ a_old,
                                           float *__restrict__ acc, float *__restrict__ pot,
                                           uint32_t *__restrict__ nint, int accumulate, int *__restrict__ err) {
    constexpr bool EWALD = PERIODIC && !TREEPM;  // periodic tree without the mesh
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lanebit = 1u << lane;
    const unsigned lt_mask = lanebit - 1u;
    const double x0 = T.x0, y0 = T.y0, z0 = T.z0, L0 = T.L0;
    const float4 *__restrict__ bcen = T.bcen;
    const float4 *__restrict__ bcom = T.bcom;
    const int4 *__restrict__ blink = T.blink;
    const float4 *__restrict__ spart = T.spart;
    const uint64_t *__restrict__ key = T.key;
    const uint32_t *__restrict__ perm = T.perm;
    const double *__restrict__ pos = T.pos;
    const int64_t gi = g0 + lane;
    const bool valid = lane < gcount;
    const int64_t glast = g0 + gcount - 1;
    const uint32_t s = sidx ? sidx[valid ? gi : g0] : (uint32_t)(valid ? gi : g0);
    const uint32_t s_first = sidx ? sidx[g0] : (uint32_t)g0;
    const uint32_t s_last = sidx ? sidx[glast] : (uint32_t)glast;
    const uint32_t out = slot ? slot[valid ? gi : g0] : perm[s];

    // group frame: centre of the smallest key cell holding the first and last particle
    const uint64_t kf = key[s_first], kl = key[s_last];
    const uint64_t kx = kf ^ kl;
    const int glevel = kx ? min((__clzll(kx) - 1) / 3, kMaxLevel) : kMaxLevel;
    const uint64_t gpre = kf >> (3 * (kMaxLevel - glevel));
    const double ghalf = ldexp(L0, -(glevel + 1));
    double gcx_d = (double)(2 * (uint64_t)compact3w(gpre) + 1) * ghalf;
    double gcy_d = (double)(2 * (uint64_t)compact3w(gpre >> 1) + 1) * ghalf;
    double gcz_d = (double)(2 * (uint64_t)compact3w(gpre >> 2) + 1) * ghalf;
    if (!PERIODIC && k.plain) {  // the plain FP32 form: absolute FP32 coordinates
        gcx_d = -x0;
        gcy_d = -y0;
        gcz_d = -z0;
    }
    const uint32_t j = perm[s];
    const double dxo = pos[3 * j] - (x0 + gcx_d), dyo = pos[3 * j + 1] - (y0 + gcy_d),
                 dzo = pos[3 * j + 2] - (z0 + gcz_d);
    float xox = (float)dxo, xoy = (float)dyo, xoz = (float)dzo;
    float thr = k.thr_const;
    if (RELATIVE)
        thr = valid ? k.alpha_over_G * fabsf(a_old[out]) : 0.0f;
    const float hi = VARH ? __ldg(&T.psoft[s]) : 0.0f;  // this particle's spline support
    float hmin_g = VARH && valid ? hi : __int_as_float(0x7f800000);
    if (VARH)
        for (int o = 16; o > 0; o >>= 1)
            hmin_g = fminf(hmin_g, __shfl_xor_sync(FULL, hmin_g, o));

    // group bounding box and criterion thresholds over the valid lanes
    const float inf = __int_as_float(0x7f800000);
    float lox, loy, loz, hix, hiy, hiz;
    auto bounding_box = [&]() {
        lox = valid ? xox : inf, loy = valid ? xoy : inf, loz = valid ? xoz : inf;
        hix = valid ? xox : -inf, hiy = valid ? xoy : -inf, hiz = valid ? xoz : -inf;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lox = fminf(lox, __shfl_xor_sync(FULL, lox, o));
            loy = fminf(loy, __shfl_xor_sync(FULL, loy, o));
            loz = fminf(loz, __shfl_xor_sync(FULL, loz, o));
            hix = fmaxf(hix, __shfl_xor_sync(FULL, hix, o));
            hiy = fmaxf(hiy, __shfl_xor_sync(FULL, hiy, o));
            hiz = fmaxf(hiz, __shfl_xor_sync(FULL, hiz, o));
        }
    };
    bounding_box();
    if (!PERIODIC && !k.plain) {
        // Open boundaries: move the frame centre to the middle of the group's
        // bounding box, on the grid of the node centres (2^-22 L0, so that
        // node-to-frame offsets stay exact in FP32), and take the offsets
        // again in FP64.  The key cell can be far larger than the group (a
        // group across a coarse cell boundary, or inside a depth-capped cell
        // much wider than its particles' separations).
        const float q = (float)ldexp(L0, -22), iq = (float)ldexp(1.0 / L0, 22);  // powers of two
        const float sx = q * rintf(0.5f * (lox + hix) * iq), sy = q * rintf(0.5f * (loy + hiy) * iq),
                    sz = q * rintf(0.5f * (loz + hiz) * iq);
        gcx_d += (double)sx;
        gcy_d += (double)sy;
        gcz_d += (double)sz;
        xox = (float)(dxo - (double)sx);
        xoy = (float)(dyo - (double)sy);
        xoz = (float)(dzo - (double)sz);
        bounding_box();
    }
    const float gcx = (float)gcx_d, gcy = (float)gcy_d, gcz = (float)gcz_d;
    float tmin = valid ? thr : inf, tmax = valid ? thr : 0.0f;
    if (RELATIVE) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tmin = fminf(tmin, __shfl_xor_sync(FULL, tmin, o));
            tmax = fmaxf(tmax, __shfl_xor_sync(FULL, tmax, o));
        }
    }
    bool wide = false;
    if (PERIODIC) {
        const float ext = fmaxf(fmaxf(fmaxf(-lox, hix), fmaxf(-loy, hiy)), fmaxf(-loz, hiz));
        wide = ext > 0.125f * k.box;
    }
    const unsigned valid_mask = __ballot_sync(FULL, valid);

    float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
    float4 ec = make_float4(0.f, 0.f, 0.f, 0.f);  // compensation of the Ewald sums
    uint32_t cnt = 0;
    put_part_entry(sh, lane, make_float4(xox, xoy, xoz, thr));  // read by the transposed decisions
    if (lane == 0) {
        sh.stack[0] = make_uint2(0u, valid_mask);  // the root, breadth-first index 0
        sh.scount[0] = 1;
    }
    int sn = 1, nf = 0, np = 0, nl = 0, nu = 0;
    __syncwarp();
    for (;;) {
        // once the stack and the undecided queue are empty, the queued
        // monopoles and leaves are swept a last time and the walk ends (one
        // copy of each sweep serves both)
        const bool done = sn == 0 && nu == 0;
        if (!done) {
        // nodes waiting for per-particle decisions go first once a full batch
        // waits (and the stack has room for what they may open), when the
        // stack is empty, or when the queue could not take another batch
        const int room = SH::kStack - 53 - sn;
        const bool resolve = nu > 0 && (sn == 0 || (nu >= 32 && room >= 32) || nu > kUndCap - 33);
        int cls = kNone;
        uint32_t nmask = 0;  // lanes that need the node (resolution: lanes that open it)
        uint32_t amask = 0;  // resolution: lanes that accept the node
        float4 C = make_float4(0.f, 0.f, 0.f, 0.f), O = C;
        int4 Lk = make_int4(0, 0, 0, 0);
        float dcx = 0.f, dcy = 0.f, dcz = 0.f;
        float hsig = 0.0f;  // the node's largest softening, negative when mixed
        uint32_t node = 0;
        if (resolve) {
            // ---- one waiting node per lane, decided for every particle of the group
            const int nr = min(min(nu, 32), max(room, 1));
            uint2 U = make_uint2(0u, 0u);
            if (lane < nr) {
                U = sh.und[nu - nr + lane];
                C = __ldg(&bcen[U.x]);
                O = __ldg(&bcom[U.x]);
                Lk = __ldg(&blink[U.x]);
                if (VARH)
                    hsig = __ldg(&T.bsoft[U.x]);
            }
            nu -= nr;
            const float dx = C.x - gcx, dy = C.y - gcy, dz = C.z - gcz;  // exact
            const float L = C.w;
            const float q = RELATIVE ? O.w * L * L : L * L;
            const float gl = 0.6f * L;
            unsigned om = 0u, am = 0u;
            if (!PERIODIC && !TREEPM && !VARH) {
                // particle pairs through the two-wide FP32 instructions; each
                // element is rounded as in the scalar form, so the decisions
                // are the same bits
                const float2 ndx = make_float2(-dx, -dx), ndy = make_float2(-dy, -dy), ndz = make_float2(-dz, -dz);
                const float2 ox = make_float2(O.x, O.x), oy = make_float2(O.y, O.y), oz = make_float2(O.z, O.z);
                const float2 m1 = make_float2(-1.0f, -1.0f);
                const bool guard_on = k.box_guard != 0;
                unsigned uy = U.y;  // lane bits still to decide, particle pair i in bits 0-1
#pragma unroll 2
                for (int i = 0; i < 16; i++, uy >>= 2) {
                    const float4 XY = sh.pxy[i], ZT = sh.pzt[i];
                    const float2 px = __fadd2_rn(make_float2(XY.x, XY.y), ndx);
                    const float2 py = __fadd2_rn(make_float2(XY.z, XY.w), ndy);
                    const float2 pz = __fadd2_rn(make_float2(ZT.x, ZT.y), ndz);
                    const float2 rx = __ffma2_rn(px, m1, ox), ry = __ffma2_rn(py, m1, oy), rz = __ffma2_rn(pz, m1, oz);
                    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
                    float2 t = __fmul2_rn(make_float2(ZT.z, ZT.w), r2);
                    if (RELATIVE)
                        t = __fmul2_rn(t, r2);
                    const bool g0 = guard_on && fmaxf(fabsf(px.x), fmaxf(fabsf(py.x), fabsf(pz.x))) <= gl;
                    const bool g1 = guard_on && fmaxf(fabsf(px.y), fmaxf(fabsf(py.y), fabsf(pz.y))) <= gl;
                    const bool o0 = g0 || q > t.x, o1 = g1 || q > t.y;
                    const unsigned b0 = 1u << (2 * i), b1 = 2u << (2 * i);
                    if (uy & 1u)
                        o0 ? (om |= b0) : (am |= b0);
                    if (uy & 2u)
                        o1 ? (om |= b1) : (am |= b1);
                }
            } else {
            const unsigned umask = __reduce_or_sync(FULL, U.y);
            for (unsigned m = umask; m; m &= m - 1u) {
                const int p = __ffs(m) - 1;
                const float4 P = part_entry(sh, p);
                const bool act = (U.y >> p) & 1u;
                float px = P.x - dx, py = P.y - dy, pz = P.z - dz;
                if (PERIODIC) {
                    px = wrap_min_image(px, k);
                    py = wrap_min_image(py, k);
                    pz = wrap_min_image(pz, k);
                }
                float rx = O.x - px, ry = O.y - py, rz = O.z - pz;
                if (PERIODIC && (EWALD || L > k.bigL)) {
                    rx = wrap_min_image(rx, k);
                    ry = wrap_min_image(ry, k);
                    rz = wrap_min_image(rz, k);
                }
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                bool far = false;
                if (TREEPM) {
                    const float ex = fmaxf(fabsf(px) - 0.5f * L, 0.0f), ey = fmaxf(fabsf(py) - 0.5f * L, 0.0f),
                                ez = fmaxf(fabsf(pz) - 0.5f * L, 0.0f);
                    far = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > k.rcut2;
                }
                const bool guard = k.box_guard && fabsf(px) <= gl && fabsf(py) <= gl && fabsf(pz) <= gl;
                bool crit = RELATIVE ? (q > P.w * r2 * r2) : (q > P.w * r2);
                if (VARH) {  // Sec. 3.2: a node of mixed softenings is opened inside its largest one
                    const float hp = __shfl_sync(FULL, hi, p);
                    crit = crit || (hsig < 0.0f && hp < -hsig && r2 < hsig * hsig);
                }
                const unsigned b = 1u << p;
                if (act && !far)
                    (guard || crit) ? (om |= b) : (am |= b);
            }
            }
            node = U.x;
            nmask = om;
            amask = am;
            dcx = dx;
            dcy = dy;
            dcz = dz;
            if (PERIODIC) {
                dcx = wrap_min_image(dcx, k);
                dcy = wrap_min_image(dcy, k);
                dcz = wrap_min_image(dcz, k);
            }
            cls = (lane < nr) ? kMixed : kNone;
        } else {
            // ---- take up to 32 candidates from the top child ranges
            const int cap = sn > SH::kSafe ? 1 : 32;
            const int idx = sn - 1 - lane;
            uint2 R = make_uint2(0u, 0u);
            int c = 0;
            if (idx >= 0) {
                R = sh.stack[idx];
                c = sh.scount[idx];
            }
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o)
                    incl += v;
            }
            const int excl = incl - c;
            const bool take = idx >= 0 && c > 0 && excl < cap;
            const bool whole = take && incl <= cap;
            const int ntake = take ? min(c, cap - excl) : 0;
            const int nwhole = __popc(__ballot_sync(FULL, whole));
            const int ncand = min(__shfl_sync(FULL, incl, 31), cap);
            // candidate `lane` comes from the range r whose prefix sums
            // bracket it (binary search over the nondecreasing incl)
            int r = 0;
#pragma unroll
            for (int b = 16; b > 0; b >>= 1)
                if (__shfl_sync(FULL, incl, r + b - 1) <= lane)
                    r += b;
            const uint32_t cnode = __shfl_sync(FULL, R.x, r) + (uint32_t)(lane - __shfl_sync(FULL, excl, r));
            const uint32_t cmask = __shfl_sync(FULL, R.y, r);
            if (take && !whole) {  // the partly taken range stays on top
                sh.stack[idx].x = R.x + (uint32_t)ntake;
                sh.scount[idx] = (uint8_t)(c - ntake);
            }
            sn -= nwhole;
            __syncwarp();

            // ---- one candidate per lane: decide for the whole group
            if (lane < ncand) {
                node = cnode;
                nmask = cmask;
                C = __ldg(&bcen[cnode]);
                O = __ldg(&bcom[cnode]);
                Lk = __ldg(&blink[cnode]);
                if (VARH)
                    hsig = __ldg(&T.bsoft[cnode]);
                cls = classify_group<PERIODIC, RELATIVE, TREEPM, VARH>(C, O, gcx, gcy, gcz, lox, loy, loz, hix, hiy,
                                                                       hiz, tmin, tmax, wide, hsig, hmin_g, k, dcx,
                                                                       dcy, dcz);
            }
            // nodes the bounds cannot decide wait for the per-particle decisions
            const unsigned bm = __ballot_sync(FULL, cls == kMixed);
            if (cls == kMixed)
                sh.und[nu + __popc(bm & lt_mask)] = make_uint2(node, nmask);
            nu += __popc(bm);
            if (cls == kAccept) {
                amask = nmask;
                nmask = 0u;
            } else if (cls != kOpen) {
                nmask = 0u;
            }
        }
        __syncwarp();
        // ---- queue what the lanes accept and open: amask = lanes that take the
        // node's monopole, nmask = lanes that open it
        const bool is_leaf = Lk.y == 0;
        // pair vectors are wrapped per lane when the group-centred image may
        // not be the particle's nearest one, and always for the Ewald table
        const bool wrapf = PERIODIC && (EWALD || wide || C.w > k.bigL);
        const bool e_acc = amask != 0u;
        const bool e_full = e_acc && amask == valid_mask;
        const unsigned bf = __ballot_sync(FULL, e_full);
        const unsigned bq = __ballot_sync(FULL, e_acc && !e_full);
        if (e_acc) {
            const int at = e_full ? nf + __popc(bf & lt_mask) : kNodeCap - 1 - np - __popc(bq & lt_mask);
            put_node_entry(sh, at, make_float4(dcx + O.x, dcy + O.y, dcz + O.z, O.w));
            sh.nmask[at] = amask;
            if (PERIODIC)
                sh.nwrap[at] = wrapf ? 1 : 0;
            if (VARH)
                sh.nsoft[at] = fabsf(hsig);
        }
        nf += __popc(bf);
        np += __popc(bq);
        const bool e_leaf = nmask != 0u && is_leaf, e_push = nmask != 0u && !is_leaf;
        const unsigned bl = __ballot_sync(FULL, e_leaf);
        if (e_leaf) {
            const int at = nl + __popc(bl & lt_mask);
            sh.lsrc[at] = make_float4(dcx, dcy, dcz, __int_as_float(Lk.z));
            sh.lmeta[at] = make_uint2(nmask, (wrapf ? kLeafWrap : 0u) | (uint32_t)Lk.w);
        }
        nl += __popc(bl);
        const unsigned bp = __ballot_sync(FULL, e_push);
        if (e_push) {
            const int at = sn + __popc(bp & lt_mask);
            if (at < SH::kStack) {
                sh.stack[at] = make_uint2((uint32_t)Lk.x, nmask);
                sh.scount[at] = (uint8_t)Lk.y;
            } else {
                atomicOr(err, 2);
            }
        }
        sn = min(sn + __popc(bp), SH::kStack);
        __syncwarp();
        }
        if (done || nf + np >= kNodeFlush) {
            sweep_full<PERIODIC, TREEPM, VARH>(sh, nf, xox, xoy, xoz, hi, k, ax, ay, az, ph, ec);
            sweep_partial<PERIODIC, TREEPM, VARH>(sh, np, lanebit, xox, xoy, xoz, hi, k, ax, ay, az, ph, cnt, ec);
            cnt += valid ? (uint32_t)nf : 0u;
            nf = np = 0;
        }
        if (done || nl >= kLeafFlush) {
            sweep_leaves<PERIODIC, TREEPM, VARH>(sh, nl, lanebit, s, xox, xoy, xoz, hi, spart, T.psoft, k, ax, ay, az,
                                                 ph, cnt, ec);
            nl = 0;
        }
        if (done)
            break;
        __syncwarp();
    }
    if (!valid)
        return;
    if (EWALD)  // the particle's own images and the background
        ph = fmaf(__ldg(&spart[s]).w * k.eps, k.ephi0, ph);
    const float G = k.G;
    if (accumulate) {
        acc[3 * (size_t)out] += G * ax;
        acc[3 * (size_t)out + 1] += G * ay;
        acc[3 * (size_t)out + 2] += G * az;
        if (pot)
            pot[out] += G * ph;
    } else {
        acc[3 * (size_t)out] = G * ax;
        acc[3 * (size_t)out + 1] = G * ay;
        acc[3 * (size_t)out + 2] = G * az;
        if (pot)
            pot[out] = G * ph;
    }
    if (nint)
        nint[out] = cnt;
}


// Walks a chunk of consecutive active particles: in one frame, or, when it
// is spread out (chunk_cuts), run by run, each run in its own frame.
template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH, class SH>
__device__ __forceinline__ void walk_runs_of_chunk(const TreeView &T, const WalkConsts &k, SH &sh,
                                                   const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                                                   int64_t g0, int gcount, const float *__restrict__ a_old,
                                                   float *__restrict__ acc, float *__restrict__ pot,
                                                   uint32_t *__restrict__ nint, int accumulate, int *__restrict__ err) {
    // a periodic box bounds every frame; the plain FP32 form has one frame
    unsigned cut = (PERIODIC || k.plain) ? 0u : chunk_cuts(T.key, sidx, g0, gcount);
    int start = 0;
    for (;;) {
        const int end = cut ? __ffs(cut) : gcount;
        group_walk<PERIODIC, RELATIVE, TREEPM, VARH>(T, k, sh, sidx, slot, g0 + start, end - start, a_old, acc, pot,
                                                     nint, accumulate, err);
        if (!cut)
            break;
        cut &= cut - 1u;
        start = end;
        __syncwarp();
    }
}

// One warp per group of `gsize` consecutive active particles.  Seven blocks
// of four warps per SM: the register cap (72) that keeps the paired FP32
// sweeps and decisions free of spills (measured against caps of 64 and none).
template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH>
__global__ void __launch_bounds__(kGroupWarps * 32, 7)
    k_walk_group(TreeView T, const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                 const float *__restrict__ a_old, int64_t n_act, int gsize, WalkConsts k, float *__restrict__ acc,
                 float *__restrict__ pot, uint32_t *__restrict__ nint, int accumulate, int *__restrict__ err) {
    using SH = GroupSharedT<kStackCap, VARH, PERIODIC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = reinterpret_cast<SH *>(smem_raw)[threadIdx.x >> 5];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t g0 = warp * gsize;
    if (g0 >= n_act)
        return;  // whole warp
    const int gcount = (int)min((int64_t)gsize, n_act - g0);
    walk_runs_of_chunk<PERIODIC, RELATIVE, TREEPM, VARH>(T, k, sh, sidx, slot, g0, gcount, a_old, acc, pot, nint,
                                                         accumulate, err);
}

// The runs of cut chunks, one warp per run.
template <bool PERIODIC, bool RELATIVE, bool TREEPM, bool VARH>
__global__ void __launch_bounds__(kGroupWarps * 32)
    k_walk_runs(TreeView T, const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                const float *__restrict__ a_old, const uint2 *__restrict__ runs, const unsigned *__restrict__ nruns,
                WalkConsts k, float *__restrict__ acc, float *__restrict__ pot, uint32_t *__restrict__ nint,
                int accumulate, int *__restrict__ err) {
    using SH = GroupSharedT<kStackCap, VARH, PERIODIC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = reinterpret_cast<SH *>(smem_raw)[threadIdx.x >> 5];
    const unsigned total = *nruns;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const uint2 R = runs[w];
        group_walk<PERIODIC, RELATIVE, TREEPM, VARH>(T, k, sh, sidx, slot, R.x, (int)R.y, a_old, acc, pot, nint,
                                                     accumulate, err);
        __syncwarp();
    }
}

// ======================================================================
// 64-particle groups (the batched walk: open boundaries, one softening
// length).  Lane l holds particles l and l + 32 of the group; lane masks are
// 64-bit (bit p = particle p).  Candidates, bounds, undecided nodes and
// queues work as in group_walk; each pair term runs through the two-wide
// FP32 instructions over the lane's two particles, so every node record the
// warp reads serves 64 particles.
// ======================================================================
template <int STACK>
struct GroupShared64 {
    static constexpr int kStack = STACK;
    static constexpr int kSafe = STACK - 64;  // above this, take one candidate at a time
    uint32_t schild[STACK];                  // first child of a range
    unsigned long long smask[STACK];         // particles that need it
    uint8_t scount[STACK];
    float4 nsrc[kNodeCap];                   // accepted node: centre of mass (group frame) + mass
    unsigned long long nmask[kNodeCap];
    float4 lsrc[kLeafCap];                   // opened leaf: centre (group frame) + first particle
    unsigned long long lmask[kLeafCap];
    uint32_t lcount[kLeafCap];
    uint32_t unode[kUndCap];                 // nodes the bounds left undecided
    unsigned long long umask[kUndCap];
    float4 pxy[32];                          // the particles by pairs (2i, 2i + 1): (x, x', y, y')
    float4 pzt[32];                          // (z, z', t, t')
};

template <class SH>
__device__ __forceinline__ void put_part64(SH &sh, int p, float x, float y, float z, float t) {
    float *a = reinterpret_cast<float *>(&sh.pxy[p >> 1]);
    float *b = reinterpret_cast<float *>(&sh.pzt[p >> 1]);
    const int o = p & 1;
    a[o] = x;
    a[2 + o] = y;
    b[o] = z;
    b[2 + o] = t;
}

__device__ __forceinline__ unsigned long long ballot64(bool lo, bool hi) {
    return (unsigned long long)__ballot_sync(0xffffffffu, lo) |
           ((unsigned long long)__ballot_sync(0xffffffffu, hi) << 32);
}

// Walks the tree for the group of gcount <= 64 active particles at positions
// [g0, g0 + gcount) of the sorted active list, two per lane.
template <bool RELATIVE, class SH>
__device__ __forceinline__ void group_walk64(const TreeView &T, const WalkConsts &k, SH &sh,
                                             const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                                             int64_t g0, int gcount, const float *__restrict__ a_old,
                                             float *__restrict__ acc, float *__restrict__ pot,
                                             uint32_t *__restrict__ nint, int *__restrict__ err) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const double x0 = T.x0, y0 = T.y0, z0 = T.z0, L0 = T.L0;
    const float4 *__restrict__ bcen = T.bcen;
    const float4 *__restrict__ bcom = T.bcom;
    const int4 *__restrict__ blink = T.blink;
    const float4 *__restrict__ spart = T.spart;
    const uint32_t *__restrict__ perm = T.perm;
    const double *__restrict__ pos = T.pos;
    const bool v0 = lane < gcount, v1 = lane + 32 < gcount;
    const int64_t glast = g0 + gcount - 1;
    const int64_t i0 = v0 ? g0 + lane : g0, i1 = v1 ? g0 + 32 + lane : g0;
    const uint32_t s0 = sidx ? sidx[i0] : (uint32_t)i0, s1 = sidx ? sidx[i1] : (uint32_t)i1;
    const uint32_t o0 = slot ? slot[i0] : perm[s0], o1 = slot ? slot[i1] : perm[s1];
    const uint32_t s_first = sidx ? sidx[g0] : (uint32_t)g0;
    const uint32_t s_last = sidx ? sidx[glast] : (uint32_t)glast;

    // frame: the key cell of the first and last particle, moved to the middle
    // of the group's bounding box on the grid of the node centres (as in
    // group_walk)
    const uint64_t kf = T.key[s_first], kl = T.key[s_last];
    const uint64_t kx = kf ^ kl;
    const int glevel = kx ? min((__clzll(kx) - 1) / 3, kMaxLevel) : kMaxLevel;
    const uint64_t gpre = kf >> (3 * (kMaxLevel - glevel));
    const double ghalf = ldexp(L0, -(glevel + 1));
    double gc[3] = {(double)(2 * (uint64_t)compact3w(gpre) + 1) * ghalf,
                    (double)(2 * (uint64_t)compact3w(gpre >> 1) + 1) * ghalf,
                    (double)(2 * (uint64_t)compact3w(gpre >> 2) + 1) * ghalf};
    const double org[3] = {x0, y0, z0};
    if (k.plain)  // the plain FP32 form: absolute FP32 coordinates
        for (int a = 0; a < 3; a++)
            gc[a] = -org[a];
    const uint32_t j0 = perm[s0], j1 = perm[s1];
    double d0[3], d1[3];
    float p0[3], p1[3];
    for (int a = 0; a < 3; a++) {
        d0[a] = pos[3 * j0 + a] - (org[a] + gc[a]);
        d1[a] = pos[3 * j1 + a] - (org[a] + gc[a]);
        p0[a] = (float)d0[a];
        p1[a] = (float)d1[a];
    }
    const float inf = __int_as_float(0x7f800000);
    float lo[3], hi[3];
    auto bounding_box = [&]() {
        for (int a = 0; a < 3; a++) {
            lo[a] = fminf(v0 ? p0[a] : inf, v1 ? p1[a] : inf);
            hi[a] = fmaxf(v0 ? p0[a] : -inf, v1 ? p1[a] : -inf);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(FULL, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULL, hi[a], o));
            }
        }
    };
    bounding_box();
    if (!k.plain) {
        const float q = (float)ldexp(L0, -22), iq = (float)ldexp(1.0 / L0, 22);
        for (int a = 0; a < 3; a++) {
            const float sa = q * rintf(0.5f * (lo[a] + hi[a]) * iq);
            gc[a] += (double)sa;
            p0[a] = (float)(d0[a] - (double)sa);
            p1[a] = (float)(d1[a] - (double)sa);
        }
        bounding_box();
    }
    const float gcx = (float)gc[0], gcy = (float)gc[1], gcz = (float)gc[2];
    float t0 = k.thr_const, t1 = k.thr_const;
    if (RELATIVE) {
        t0 = v0 ? k.alpha_over_G * fabsf(a_old[o0]) : 0.0f;
        t1 = v1 ? k.alpha_over_G * fabsf(a_old[o1]) : 0.0f;
    }
    float tmin = fminf(v0 ? t0 : inf, v1 ? t1 : inf), tmax = fmaxf(v0 ? t0 : 0.0f, v1 ? t1 : 0.0f);
    if (RELATIVE) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tmin = fminf(tmin, __shfl_xor_sync(FULL, tmin, o));
            tmax = fmaxf(tmax, __shfl_xor_sync(FULL, tmax, o));
        }
    }
    const unsigned long long valid_mask = ballot64(v0, v1);
    put_part64(sh, lane, p0[0], p0[1], p0[2], t0);
    put_part64(sh, lane + 32, p1[0], p1[1], p1[2], t1);
    // the lane's two particles as pairs for the two-wide instructions
    const float2 nx = make_float2(-p0[0], -p1[0]), ny = make_float2(-p0[1], -p1[1]), nz = make_float2(-p0[2], -p1[2]);
    float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx, sp = sx;  // acceleration and potential sums
    uint32_t c0 = 0, c1 = 0;                                       // interaction counts
    if (lane == 0) {
        sh.schild[0] = 0u;  // the root, breadth-first index 0
        sh.smask[0] = valid_mask;
        sh.scount[0] = 1;
    }
    int sn = 1, nf = 0, np = 0, nl = 0, nu = 0;
    __syncwarp();
    for (;;) {
        const bool done = sn == 0 && nu == 0;
        if (!done) {
            const int room = SH::kStack - 53 - sn;
            const bool resolve = nu > 0 && (sn == 0 || (nu >= 32 && room >= 32) || nu > kUndCap - 33);
            int cls = kNone;
            unsigned long long nmask = 0ull, amask = 0ull;
            float4 C = make_float4(0.f, 0.f, 0.f, 0.f), O = C;
            int4 Lk = make_int4(0, 0, 0, 0);
            float dcx = 0.f, dcy = 0.f, dcz = 0.f;
            uint32_t node = 0;
            if (resolve) {
                // ---- one waiting node per lane, decided for all 64 particles
                const int nr = min(min(nu, 32), max(room, 1));
                unsigned long long um = 0ull;
                if (lane < nr) {
                    node = sh.unode[nu - nr + lane];
                    um = sh.umask[nu - nr + lane];
                    C = __ldg(&bcen[node]);
                    O = __ldg(&bcom[node]);
                    Lk = __ldg(&blink[node]);
                }
                nu -= nr;
                dcx = C.x - gcx;
                dcy = C.y - gcy;
                dcz = C.z - gcz;  // exact
                const float L = C.w;
                const float q = RELATIVE ? O.w * L * L : L * L;
                const float gl = 0.6f * L;
                const float2 ndx = make_float2(-dcx, -dcx), ndy = make_float2(-dcy, -dcy), ndz = make_float2(-dcz, -dcz);
                const float2 ox = make_float2(O.x, O.x), oy = make_float2(O.y, O.y), oz = make_float2(O.z, O.z);
                const float2 m1 = make_float2(-1.0f, -1.0f);
                const bool guard_on = k.box_guard != 0;
                unsigned long long om = 0ull, am = 0ull, uy = um;
#pragma unroll 2
                for (int i = 0; i < 32; i++, uy >>= 2) {
                    const float4 XY = sh.pxy[i], ZT = sh.pzt[i];
                    const float2 px = __fadd2_rn(make_float2(XY.x, XY.y), ndx);
                    const float2 py = __fadd2_rn(make_float2(XY.z, XY.w), ndy);
                    const float2 pz = __fadd2_rn(make_float2(ZT.x, ZT.y), ndz);
                    const float2 rx = __ffma2_rn(px, m1, ox), ry = __ffma2_rn(py, m1, oy), rz = __ffma2_rn(pz, m1, oz);
                    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
                    float2 t = __fmul2_rn(make_float2(ZT.z, ZT.w), r2);
                    if (RELATIVE)
                        t = __fmul2_rn(t, r2);
                    const bool g0b = guard_on && fmaxf(fabsf(px.x), fmaxf(fabsf(py.x), fabsf(pz.x))) <= gl;
                    const bool g1b = guard_on && fmaxf(fabsf(px.y), fmaxf(fabsf(py.y), fabsf(pz.y))) <= gl;
                    const bool oa = g0b || q > t.x, ob = g1b || q > t.y;
                    const unsigned long long b0 = 1ull << (2 * i), b1 = 2ull << (2 * i);
                    if (uy & 1ull)
                        oa ? (om |= b0) : (am |= b0);
                    if (uy & 2ull)
                        ob ? (om |= b1) : (am |= b1);
                }
                nmask = om;
                amask = am;
                cls = lane < nr ? kMixed : kNone;
            } else {
                // ---- up to 32 candidates from the top child ranges
                const int cap = sn > SH::kSafe ? 1 : 32;
                const int idx = sn - 1 - lane;
                uint32_t rchild = 0u;
                unsigned long long rmask = 0ull;
                int c = 0;
                if (idx >= 0) {
                    rchild = sh.schild[idx];
                    rmask = sh.smask[idx];
                    c = sh.scount[idx];
                }
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o)
                        incl += v;
                }
                const int excl = incl - c;
                const bool take = idx >= 0 && c > 0 && excl < cap;
                const bool whole = take && incl <= cap;
                const int ntake = take ? min(c, cap - excl) : 0;
                const int nwhole = __popc(__ballot_sync(FULL, whole));
                const int ncand = min(__shfl_sync(FULL, incl, 31), cap);
                int r = 0;
#pragma unroll
                for (int b = 16; b > 0; b >>= 1)
                    if (__shfl_sync(FULL, incl, r + b - 1) <= lane)
                        r += b;
                const uint32_t cnode = __shfl_sync(FULL, rchild, r) + (uint32_t)(lane - __shfl_sync(FULL, excl, r));
                const unsigned long long cmask = __shfl_sync(FULL, rmask, r);
                if (take && !whole) {  // the partly taken range stays on top
                    sh.schild[idx] = rchild + (uint32_t)ntake;
                    sh.scount[idx] = (uint8_t)(c - ntake);
                }
                sn -= nwhole;
                __syncwarp();
                if (lane < ncand) {
                    node = cnode;
                    nmask = cmask;
                    C = __ldg(&bcen[cnode]);
                    O = __ldg(&bcom[cnode]);
                    Lk = __ldg(&blink[cnode]);
                    cls = classify_group<false, RELATIVE, false, false>(C, O, gcx, gcy, gcz, lo[0], lo[1], lo[2], hi[0],
                                                                        hi[1], hi[2], tmin, tmax, false, 0.0f, inf, k,
                                                                        dcx, dcy, dcz);
                }
                const unsigned bm = __ballot_sync(FULL, cls == kMixed);
                if (cls == kMixed) {
                    const int at = nu + __popc(bm & lt_mask);
                    sh.unode[at] = node;
                    sh.umask[at] = nmask;
                }
                nu += __popc(bm);
                if (cls == kAccept) {
                    amask = nmask;
                    nmask = 0ull;
                } else if (cls != kOpen) {
                    nmask = 0ull;
                }
            }
            __syncwarp();
            // ---- queue what the particles accept and open
            const bool is_leaf = Lk.y == 0;
            const bool e_acc = amask != 0ull;
            const bool e_full = e_acc && amask == valid_mask;
            const unsigned bf = __ballot_sync(FULL, e_full);
            const unsigned bq = __ballot_sync(FULL, e_acc && !e_full);
            if (e_acc) {
                const int at = e_full ? nf + __popc(bf & lt_mask) : kNodeCap - 1 - np - __popc(bq & lt_mask);
                sh.nsrc[at] = make_float4(dcx + O.x, dcy + O.y, dcz + O.z, O.w);
                sh.nmask[at] = amask;
            }
            nf += __popc(bf);
            np += __popc(bq);
            const bool e_leaf = nmask != 0ull && is_leaf, e_push = nmask != 0ull && !is_leaf;
            const unsigned bl = __ballot_sync(FULL, e_leaf);
            if (e_leaf) {
                const int at = nl + __popc(bl & lt_mask);
                sh.lsrc[at] = make_float4(dcx, dcy, dcz, __int_as_float(Lk.z));
                sh.lmask[at] = nmask;
                sh.lcount[at] = (uint32_t)Lk.w;
            }
            nl += __popc(bl);
            const unsigned bp = __ballot_sync(FULL, e_push);
            if (e_push) {
                const int at = sn + __popc(bp & lt_mask);
                if (at < SH::kStack) {
                    sh.schild[at] = (uint32_t)Lk.x;
                    sh.smask[at] = nmask;
                    sh.scount[at] = (uint8_t)Lk.y;
                } else {
                    atomicOr(err, 2);
                }
            }
            sn = min(sn + __popc(bp), SH::kStack);
            __syncwarp();
        }
        if (done || nf + np >= kNodeFlush) {
            // ---- monopoles: the lane's two particles per entry; a particle
            // outside the entry's mask adds zero mass; every entry first at
            // max(r, h), then the h-terms of entries inside h replaced
            float rmin = inf;
            const int e0 = kNodeCap - np;
            for (int pass = 0; pass < 2; pass++) {
                const int ea = pass ? e0 : 0, eb = pass ? kNodeCap : nf;
#pragma unroll 2
                for (int e = ea; e < eb; e++) {
                    const float4 A = sh.nsrc[e];
                    float2 m = make_float2(A.w, A.w);
                    if (pass) {
                        const unsigned long long M = sh.nmask[e];
                        const bool ma = (M >> lane) & 1ull, mb = (M >> (lane + 32)) & 1ull;
                        m = make_float2(ma ? A.w : 0.0f, mb ? A.w : 0.0f);
                        c0 += ma ? 1u : 0u;
                        c1 += mb ? 1u : 0u;
                    }
                    const float2 rx = __fadd2_rn(make_float2(A.x, A.x), nx);
                    const float2 ry = __fadd2_rn(make_float2(A.y, A.y), ny);
                    const float2 rz = __fadd2_rn(make_float2(A.z, A.z), nz);
                    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
                    rmin = fminf(rmin, fminf(r2.x, r2.y));
                    const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, k.h2)), rsqrtf(fmaxf(r2.y, k.h2)));
                    const float2 mr = __fmul2_rn(m, ri);
                    const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
                    sx = __ffma2_rn(mr3, rx, sx);
                    sy = __ffma2_rn(mr3, ry, sy);
                    sz = __ffma2_rn(mr3, rz, sz);
                    sp = __fadd2_rn(sp, mr);
                }
            }
            c0 += v0 ? (uint32_t)nf : 0u;
            c1 += v1 ? (uint32_t)nf : 0u;
            if (__any_sync(FULL, rmin < k.h2)) {
                for (int pass = 0; pass < 2; pass++) {
                    const int ea = pass ? e0 : 0, eb = pass ? kNodeCap : nf;
                    for (int e = ea; e < eb; e++) {
                        const float4 A = sh.nsrc[e];
                        const unsigned long long M = pass ? sh.nmask[e] : ~0ull;
                        for (int h = 0; h < 2; h++) {
                            const float *pp = h ? p1 : p0;
                            const bool mine = (M >> (lane + 32 * h)) & 1ull;
                            const float rx = A.x - pp[0], ry = A.y - pp[1], rz = A.z - pp[2];
                            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                            if (mine && r2 < k.h2) {
                                float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
                                newton_term(rx, ry, rz, k.h2, -A.w, ax, ay, az, ph);
                                pair_term<false>(rx, ry, rz, r2, A.w, k, ax, ay, az, ph);
                                if (h) {
                                    sx.y += ax; sy.y += ay; sz.y += az; sp.y -= ph;
                                } else {
                                    sx.x += ax; sy.x += ay; sz.x += az; sp.x -= ph;
                                }
                            }
                        }
                    }
                }
            }
            nf = np = 0;
        }
        if (done || nl >= kLeafFlush) {
            // ---- opened leaves, particle by particle (pairs inside h as above)
            for (int e = 0; e < nl; e++) {
                const float4 E = sh.lsrc[e];
                const unsigned long long M = sh.lmask[e];
                const bool ma = (M >> lane) & 1ull, mb = (M >> (lane + 32)) & 1ull;
                const float2 qx0 = make_float2(p0[0] - E.x, p1[0] - E.x), qy0 = make_float2(p0[1] - E.y, p1[1] - E.y),
                             qz0 = make_float2(p0[2] - E.z, p1[2] - E.z);  // particle relative to the leaf centre
                const int ja = __float_as_int(E.w), jb = ja + (int)sh.lcount[e];
                bool close = false;
                for (int jj = ja; jj < jb; jj++) {
                    const float4 P = __ldg(&spart[jj]);
                    const bool ua = ma && (uint32_t)jj != s0, ub = mb && (uint32_t)jj != s1;
                    const float2 qx = __fadd2_rn(make_float2(P.x, P.x), make_float2(-qx0.x, -qx0.y));
                    const float2 qy = __fadd2_rn(make_float2(P.y, P.y), make_float2(-qy0.x, -qy0.y));
                    const float2 qz = __fadd2_rn(make_float2(P.z, P.z), make_float2(-qz0.x, -qz0.y));
                    const float2 q2 = __ffma2_rn(qx, qx, __ffma2_rn(qy, qy, __fmul2_rn(qz, qz)));
                    close |= (ua && q2.x < k.h2) || (ub && q2.y < k.h2);
                    c0 += ua ? 1u : 0u;
                    c1 += ub ? 1u : 0u;
                    const float2 ri = make_float2(rsqrtf(fmaxf(q2.x, k.h2)), rsqrtf(fmaxf(q2.y, k.h2)));
                    const float2 mr = __fmul2_rn(make_float2(ua ? P.w : 0.0f, ub ? P.w : 0.0f), ri);
                    const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
                    sx = __ffma2_rn(mr3, qx, sx);
                    sy = __ffma2_rn(mr3, qy, sy);
                    sz = __ffma2_rn(mr3, qz, sz);
                    sp = __fadd2_rn(sp, mr);
                }
                if (__any_sync(FULL, close)) {
                    for (int jj = ja; jj < jb; jj++) {
                        const float4 P = __ldg(&spart[jj]);
                        for (int h = 0; h < 2; h++) {
                            const bool u = h ? (mb && (uint32_t)jj != s1) : (ma && (uint32_t)jj != s0);
                            const float qx = P.x - (h ? qx0.y : qx0.x), qy = P.y - (h ? qy0.y : qy0.x),
                                        qz = P.z - (h ? qz0.y : qz0.x);
                            const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                            if (u && q2 < k.h2) {
                                float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
                                newton_term(qx, qy, qz, k.h2, -P.w, ax, ay, az, ph);
                                pair_term<false>(qx, qy, qz, q2, P.w, k, ax, ay, az, ph);
                                if (h) {
                                    sx.y += ax; sy.y += ay; sz.y += az; sp.y -= ph;
                                } else {
                                    sx.x += ax; sy.x += ay; sz.x += az; sp.x -= ph;
                                }
                            }
                        }
                    }
                }
            }
            nl = 0;
        }
        if (done)
            break;
        __syncwarp();
    }
    const float G = k.G;
    if (v0) {
        acc[3 * (size_t)o0] = G * sx.x;
        acc[3 * (size_t)o0 + 1] = G * sy.x;
        acc[3 * (size_t)o0 + 2] = G * sz.x;
        if (pot)
            pot[o0] = -G * sp.x;
        if (nint)
            nint[o0] = c0;
    }
    if (v1) {
        acc[3 * (size_t)o1] = G * sx.y;
        acc[3 * (size_t)o1 + 1] = G * sy.y;
        acc[3 * (size_t)o1 + 2] = G * sz.y;
        if (pot)
            pot[o1] = -G * sp.y;
        if (nint)
            nint[o1] = c1;
    }
}

// Walks a 64-particle group in one frame, or -- when a half of it needs
// cutting (chunk_cuts) or the two halves lie far apart for their particles'
// separations -- run by run, each run in its own frame.
template <bool RELATIVE, class SH>
__device__ __forceinline__ void walk_runs_of_group64(const TreeView &T, const WalkConsts &k, SH &sh,
                                                     const uint32_t *__restrict__ sidx,
                                                     const uint32_t *__restrict__ slot, int64_t g0, int gcount,
                                                     const float *__restrict__ a_old, float *__restrict__ acc,
                                                     float *__restrict__ pot, uint32_t *__restrict__ nint,
                                                     int *__restrict__ err) {
    unsigned long long cut = 0ull;  // bit i: a run ends after particle i
    if (!k.plain && gcount > 1) {
        const int na = min(gcount, 32), nb = gcount - na;
        const unsigned ca = chunk_cuts(T.key, sidx, g0, na);
        const unsigned cb = nb > 0 ? chunk_cuts(T.key, sidx, g0 + 32, nb) : 0u;
        bool between = ca != 0u || cb != 0u;
        if (!between && nb > 0) {
            // the pair across the halves against the finest level a member
            // shares with its neighbour
            const int lane = threadIdx.x & 31;
            const int64_t ia = g0 + min(lane, na - 1), ib = g0 + 32 + min(lane, nb - 1);
            const uint64_t ka = T.key[sidx ? sidx[ia] : (uint32_t)ia], kb = T.key[sidx ? sidx[ib] : (uint32_t)ib];
            const uint64_t kan = __shfl_down_sync(0xffffffffu, ka, 1), kbn = __shfl_down_sync(0xffffffffu, kb, 1);
            int fin = max(lane + 1 < na ? common_level(ka, kan) : -1, lane + 1 < nb ? common_level(kb, kbn) : -1);
            fin = __reduce_max_sync(0xffffffffu, fin + 1) - 1;
            const int lvb = common_level(__shfl_sync(0xffffffffu, ka, na - 1), __shfl_sync(0xffffffffu, kb, 0));
            between = fin - lvb > kFrameSpan;
        }
        if (between)
            cut = (unsigned long long)ca | (nb > 0 ? (1ull << 31) : 0ull) | ((unsigned long long)cb << 32);
    }
    int start = 0;
    for (;;) {
        const int end = cut ? __ffsll((long long)cut) : gcount;
        group_walk64<RELATIVE>(T, k, sh, sidx, slot, g0 + start, end - start, a_old, acc, pot, nint, err);
        if (!cut)
            break;
        cut &= cut - 1ull;
        start = end;
        __syncwarp();
    }
}

// One request of a batch: which tree, with which constants and criterion.
struct BatchReq {
    TreeView T;
    WalkConsts k;
    int relative;
};

// Persistent batch walk: resident warps take groups (start, count, request)
// from a device work queue until it is empty; groups of one launch may
// belong to different requests and different trees.  Compiled per candidate
// stack capacity (the plan's autotuner chooses one).
template <bool PERIODIC, bool TREEPM, int STACK>
__global__ void __launch_bounds__(kGroupWarps * 32, 7)
    k_walk_batch(const BatchReq *__restrict__ reqs, const uint4 *__restrict__ groups,
                 const unsigned *__restrict__ n_groups, unsigned *__restrict__ next, const uint32_t *__restrict__ sidx,
                 const uint32_t *__restrict__ slot, const float *__restrict__ a_old, float *__restrict__ acc,
                 float *__restrict__ pot, uint32_t *__restrict__ nint, int *__restrict__ err) {
    using SH = GroupSharedT<STACK, false, PERIODIC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = reinterpret_cast<SH *>(smem_raw)[threadIdx.x >> 5];
    // the current group's request record, read from shared memory where the
    // walk needs a field (copies in registers would crowd out the walk's own)
    __shared__ __align__(16) BatchReq breq[kGroupWarps];
    BatchReq &R = breq[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned total = *n_groups;
    for (;;) {
        unsigned g = 0;
        if (lane == 0)
            g = atomicAdd(next, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total)
            break;
        const uint4 G = groups[g];
        {
            static_assert(sizeof(BatchReq) % 4 == 0, "request records copy as words");
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&reqs[G.z]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&R);
            for (int w = lane; w < (int)(sizeof(BatchReq) / 4); w += 32)
                dst[w] = src[w];
            __syncwarp();
        }
        if (R.relative)
            walk_runs_of_chunk<PERIODIC, true, TREEPM, false>(R.T, R.k, sh, sidx, slot, G.x, (int)G.y, a_old, acc,
                                                              pot, nint, 0, err);
        else
            walk_runs_of_chunk<PERIODIC, false, TREEPM, false>(R.T, R.k, sh, sidx, slot, G.x, (int)G.y, a_old, acc,
                                                               pot, nint, 0, err);
        __syncwarp();
    }
}

// The persistent batch walk with 64-particle groups (open boundaries, one
// softening length); five blocks per SM leave the two particles' state in
// registers (96) without spilling.
template <int STACK>
__global__ void __launch_bounds__(kGroupWarps * 32, 5)
    k_walk_batch64(const BatchReq *__restrict__ reqs, const uint4 *__restrict__ groups,
                   const unsigned *__restrict__ n_groups, unsigned *__restrict__ next,
                   const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot,
                   const float *__restrict__ a_old, float *__restrict__ acc, float *__restrict__ pot,
                   uint32_t *__restrict__ nint, int *__restrict__ err) {
    using SH = GroupShared64<STACK>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = reinterpret_cast<SH *>(smem_raw)[threadIdx.x >> 5];
    __shared__ __align__(16) BatchReq breq[kGroupWarps];
    BatchReq &R = breq[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned total = *n_groups;
    for (;;) {
        unsigned g = 0;
        if (lane == 0)
            g = atomicAdd(next, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total)
            break;
        const uint4 G = groups[g];
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&reqs[G.z]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&R);
            for (int w = lane; w < (int)(sizeof(BatchReq) / 4); w += 32)
                dst[w] = src[w];
            __syncwarp();
        }
        if (R.relative)
            walk_runs_of_group64<true>(R.T, R.k, sh, sidx, slot, G.x, (int)G.y, a_old, acc, pot, nint, err);
        else
            walk_runs_of_group64<false>(R.T, R.k, sh, sidx, slot, G.x, (int)G.y, a_old, acc, pot, nint, err);
        __syncwarp();
    }
}

template <bool P, bool R, bool T, bool V>
void launch(const System *s, const WalkRequest &r, const WalkConsts &k, bool lanes, int *err, int num_sms,
            cudaStream_t st) {
    const int64_t warps = (r.n_act + 31) / 32;
    if (lanes) {
        const int64_t blocks = (warps * 32 + kWalkThreads - 1) / kWalkThreads;
        k_walk<P, R, T, V><<<(unsigned)blocks, kWalkThreads, 0, st>>>(
            s->ncen, s->ncom, s->nlink, s->spart, s->key, s->perm, s->pos, s->x0[0], s->x0[1], s->x0[2], s->L0,
            (int)s->nnodes, s->psoft, s->nsoft, r.sorted_idx, r.slot, r.a_old, r.n_act, k, r.acc, r.pot, r.nint,
            r.accumulate, r.runs, r.nruns);
        count_launch();
    }
    const size_t smem = kGroupWarps * sizeof(GroupSharedT<kStackCap, V, P>);
    TreeView tv{s->bcen, s->bcom, s->blink, s->spart, s->psoft, s->bsoft, s->key,
                s->perm, s->pos,  s->x0[0], s->x0[1],  s->x0[2], s->L0};
    if (!lanes) {
        const int64_t blocks = (warps + kGroupWarps - 1) / kGroupWarps;
        k_walk_group<P, R, T, V><<<(unsigned)blocks, kGroupWarps * 32, smem, st>>>(
            tv, r.sorted_idx, r.slot, r.a_old, r.n_act, 32, k, r.acc, r.pot, r.nint, r.accumulate, err);
        count_launch();
    } else if constexpr (!P) {
        // the lane walk hands spread-out chunks to the group walk: their runs
        // (rare: usually none, and the launch returns at once)
        const int64_t blocks = std::min<int64_t>(warps, 2 * (int64_t)num_sms);
        k_walk_runs<P, R, T, V><<<(unsigned)blocks, kGroupWarps * 32, smem, st>>>(
            tv, r.sorted_idx, r.slot, r.a_old, r.runs, r.nruns, k, r.acc, r.pot, r.nint, r.accumulate, err);
        count_launch();
    }
}

// Kernel choice: the group walk for open boundaries (with or without the
// TreePM split), the lane walk for the periodic short-range walk (there the
// cutoff sphere, a few mean spacings wide, cuts through most groups, so the
// group bounds rarely decide and the lane walk is faster).  TPM_WALK=lanes or
// group forces one for comparison; both make the same per-particle decisions.
int walk_override() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("TPM_WALK");
        v = (e && strcmp(e, "lanes") == 0) ? 1 : (e && strcmp(e, "group") == 0) ? 2 : 0;
    }
    return v;
}

WalkConsts make_consts(const System *s, const tpm_force_params *p) {
    WalkConsts k{};
    const double h = s->bp.h;
    k.h2 = (float)(h * h);
    k.hinv = (float)(1.0 / h);
    k.hinv3 = (float)(1.0 / (h * h * h));
    k.thr_const = (float)(p->theta * p->theta);
    k.alpha_over_G = (float)(p->alpha / s->bp.G);
    k.G = (float)s->bp.G;
    k.box_guard = p->box_guard ? 1 : 0;
    k.plain = p->plain_fp32 ? 1 : 0;
    k.box = (float)s->bp.box;
    k.boxinv = (float)(1.0 / s->bp.box);
    k.bigL = (float)(0.25 * s->bp.box);
    if (p->treepm) {
        const double rs = p->asmth * pm_side(s) / p->pm_n;
        const double rc = p->rcut * rs;
        k.rcut2 = (float)(rc * rc);
        k.inv2rs = (float)(1.0 / (2.0 * rs));
    }
    return k;
}

// The Ewald constants of a periodic tree without the mesh (table at unit box).
void set_ewald(WalkConsts &k, const System *s, const float4 *tab, float phi0) {
    const double L = s->bp.box;
    k.etab = tab;
    k.ent = kEwaldN;
    k.escale = (float)(2.0 * kEwaldN / L);
    k.efs = (float)(1.0 / (L * L));
    k.eps = (float)(1.0 / L);
    k.ephi0 = phi0;
}

}  // namespace

size_t batch_req_bytes() { return sizeof(BatchReq); }

void fill_batch_req(void *dst, const System *s, const tpm_force_params *p) {
    BatchReq r{};
    r.T = TreeView{s->bcen, s->bcom, s->blink, s->spart, s->psoft, s->bsoft, s->key, s->perm, s->pos, s->x0[0], s->x0[1], s->x0[2], s->L0};
    r.k = make_consts(s, p);
    r.relative = p->crit == TPM_CRIT_RELATIVE ? 1 : 0;
    memcpy(dst, &r, sizeof r);
}

template <int STACK>
int launch_walk_batch64_at(Ctx *c, const void *reqs, const uint4 *groups, const unsigned *n_groups, unsigned *next,
                           const uint32_t *sidx, const uint32_t *slot, const float *a_old, float *acc, float *pot,
                           uint32_t *nint, int *err, cudaStream_t st) {
    const size_t smem = kGroupWarps * sizeof(GroupShared64<STACK>);
    static int blocks_per_sm = 0;  // resident blocks of this variant (one persistent wave)
    if (!blocks_per_sm) {
        if (cudaFuncSetAttribute(k_walk_batch64<STACK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            set_error("64-particle groups: %zu bytes of shared memory per block are not available", smem);
            return TPM_ECUDA;
        }
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk_batch64<STACK>, kGroupWarps * 32, smem) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        blocks_per_sm = b;
    }
    k_walk_batch64<STACK><<<(unsigned)(c->num_sms * blocks_per_sm), kGroupWarps * 32, smem, st>>>(
        static_cast<const BatchReq *>(reqs), groups, n_groups, next, sidx, slot, a_old, acc, pot, nint, err);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

template <int STACK>
int launch_walk_batch_at(Ctx *c, const void *reqs, const uint4 *groups, const unsigned *n_groups, unsigned *next,
                         const uint32_t *sidx, const uint32_t *slot, const float *a_old, float *acc, float *pot,
                         uint32_t *nint, int *err, cudaStream_t st) {
    const size_t smem = kGroupWarps * sizeof(GroupSharedT<STACK, false, false>);
    static int blocks_per_sm = 0;  // resident blocks of this variant (one persistent wave)
    if (!blocks_per_sm) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk_batch<false, false, STACK>, kGroupWarps * 32,
                                                          smem) != cudaSuccess ||
            b < 1)
            b = 1;
        blocks_per_sm = b;
    }
    k_walk_batch<false, false, STACK><<<(unsigned)(c->num_sms * blocks_per_sm), kGroupWarps * 32, smem, st>>>(
        static_cast<const BatchReq *>(reqs), groups, n_groups, next, sidx, slot, a_old, acc, pot, nint, err);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

int launch_walk_batch(Ctx *c, int group_size, int stack_depth, const void *reqs, const uint4 *groups,
                      const unsigned *n_groups, unsigned *next, const uint32_t *sidx, const uint32_t *slot,
                      const float *a_old, float *acc, float *pot, uint32_t *nint, int *err, cudaStream_t st) {
    if (group_size == 64) {
        switch (stack_depth) {
        case kStackDepths[0]:
            return launch_walk_batch64_at<kStackDepths[0]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc,
                                                           pot, nint, err, st);
        case kStackDepths[1]:
            return launch_walk_batch64_at<kStackDepths[1]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc,
                                                           pot, nint, err, st);
        case kStackDepths[2]:
            return launch_walk_batch64_at<kStackDepths[2]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc,
                                                           pot, nint, err, st);
        default:
            break;
        }
    }
    switch (stack_depth) {
    case kStackDepths[0]:
        return launch_walk_batch_at<kStackDepths[0]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc, pot,
                                                     nint, err, st);
    case kStackDepths[1]:
        return launch_walk_batch_at<kStackDepths[1]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc, pot,
                                                     nint, err, st);
    case kStackDepths[2]:
        return launch_walk_batch_at<kStackDepths[2]>(c, reqs, groups, n_groups, next, sidx, slot, a_old, acc, pot,
                                                     nint, err, st);
    default:
        set_error("stack depth %d is not one of 128, 192, 256", stack_depth);
        return TPM_EINVAL;
    }
}

int walk_device(Ctx *c, const System *s, const tpm_force_params *p, const WalkRequest &r, cudaStream_t st) {
    if (r.n_act == 0)
        return TPM_OK;
    WalkConsts k = make_consts(s, p);
    const bool per = s->bp.periodic != 0, rel = p->crit == TPM_CRIT_RELATIVE, tpm = p->treepm != 0;
    if (per && !tpm) {
        const float4 *tab;
        float phi0;
        TPM_CHECK(ewald_table_for(c, !r.no_alloc, st, &tab, &phi0));
        set_ewald(k, s, tab, phi0);
    }
    const int ov = walk_override();
    const bool lanes = ov == 1 || (ov == 0 && per);
    int *err = s->err;
    if (!per && lanes) {  // the lane walk's list of cut chunks' runs: n_act entries at most
        if (!r.runs || !r.nruns) {
            set_error("internal: open-boundary lane walk without a run list");
            return TPM_EINVAL;
        }
        TPM_CUDA(cudaMemsetAsync(r.nruns, 0, sizeof(unsigned), st));
    }
    const bool varh = s->psoft != nullptr;  // per-particle softening (open boundaries only)
    if (varh && per) {
        set_error("per-particle softening is available with open boundaries");
        return TPM_EINVAL;
    }
    if (!per && !tpm)
        rel ? (varh ? launch<false, true, false, true>(s, r, k, lanes, err, c->num_sms, st)
                    : launch<false, true, false, false>(s, r, k, lanes, err, c->num_sms, st))
            : (varh ? launch<false, false, false, true>(s, r, k, lanes, err, c->num_sms, st)
                    : launch<false, false, false, false>(s, r, k, lanes, err, c->num_sms, st));
    else if (!per && tpm)
        rel ? (varh ? launch<false, true, true, true>(s, r, k, lanes, err, c->num_sms, st)
                    : launch<false, true, true, false>(s, r, k, lanes, err, c->num_sms, st))
            : (varh ? launch<false, false, true, true>(s, r, k, lanes, err, c->num_sms, st)
                    : launch<false, false, true, false>(s, r, k, lanes, err, c->num_sms, st));
    else if (tpm)
        rel ? launch<true, true, true, false>(s, r, k, lanes, err, c->num_sms, st)
            : launch<true, false, true, false>(s, r, k, lanes, err, c->num_sms, st);
    else
        rel ? launch<true, true, false, false>(s, r, k, lanes, err, c->num_sms, st)
            : launch<true, false, false, false>(s, r, k, lanes, err, c->num_sms, st);
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
