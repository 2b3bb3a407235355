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
__device__ __forceinline__ void pair_term(float rx, float ry, float rz, float r2, float m, const WalkConsts &k,
                                          float &ax, float &ay, float &az, float &ph) {
    float kf, kp;
    if (r2 >= k.h2) {
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
        const float u = r * k.hinv;
        const float u2 = u * u;
        if (u < 0.5f) {
            kf = k.hinv3 * fmaf(u2, fmaf(32.0f, u, -38.4f), 10.666666667f);
            kp = k.hinv * fmaf(u2, fmaf(u2, fmaf(6.4f, u, -9.6f), 5.333333333f), -2.8f);
        } else {
            const float iu = __fdividef(1.0f, u);
            kf = k.hinv3 * (fmaf(u, fmaf(u, fmaf(-10.666666667f, u, 38.4f), -48.0f), 21.333333333f) -
                            0.066666666667f * iu * iu * iu);
            kp = k.hinv * (fmaf(u2, fmaf(u, fmaf(u, fmaf(-2.133333333f, u, 9.6f), -16.0f), 10.666666667f), -3.2f) +
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

__device__ __forceinline__ float wrap_min_image(float d, const WalkConsts &k) {
    return fmaf(-k.box, rintf(d * k.boxinv), d);
}

template <bool PERIODIC, bool RELATIVE, bool TREEPM>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk(const float4 *__restrict__ ncen, const float4 *__restrict__ ncom, const int4 *__restrict__ nlink,
           const float4 *__restrict__ spart, const uint64_t *__restrict__ key, const uint32_t *__restrict__ perm,
           const double *__restrict__ pos, double x0, double y0, double z0, double L0, int nnodes,
           const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot, const float *__restrict__ a_old,
           int64_t n_act, WalkConsts k, float *__restrict__ acc, float *__restrict__ pot,
           uint32_t *__restrict__ nint, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane);
    if (g0 >= n_act)
        return;  // the whole warp leaves together
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
    const double gcx_d = (double)(2 * (uint64_t)compact3w(gpre) + 1) * ghalf;
    const double gcy_d = (double)(2 * (uint64_t)compact3w(gpre >> 1) + 1) * ghalf;
    const double gcz_d = (double)(2 * (uint64_t)compact3w(gpre >> 2) + 1) * ghalf;
    const float gcx = (float)gcx_d, gcy = (float)gcy_d, gcz = (float)gcz_d;
    const uint32_t j = perm[s];
    const float xox = (float)(pos[3 * j] - (x0 + gcx_d));
    const float xoy = (float)(pos[3 * j + 1] - (y0 + gcy_d));
    const float xoz = (float)(pos[3 * j + 2] - (z0 + gcz_d));

    float thr = k.thr_const;
    if (RELATIVE)
        thr = valid ? k.alpha_over_G * fabsf(a_old[out]) : 0.0f;

    float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
    uint32_t cnt = 0;
    int skip_until = valid ? 0 : 0x7fffffff;
    int n = 0;
    while (n < nnodes) {
        const float4 C = __ldg(&ncen[n]);
        const float4 O = __ldg(&ncom[n]);
        const int4 Lk = __ldg(&nlink[n]);
        const bool act = n >= skip_until;
        float dcx = C.x - gcx, dcy = C.y - gcy, dcz = C.z - gcz;  // exact
        if (PERIODIC) {
            dcx = wrap_min_image(dcx, k);
            dcy = wrap_min_image(dcy, k);
            dcz = wrap_min_image(dcz, k);
        }
        const float px = xox - dcx, py = xoy - dcy, pz = xoz - dcz;  // particle relative to node centre
        const float L = C.w;
        float rx = O.x - px, ry = O.y - py, rz = O.z - pz;  // particle -> centre of mass
        if (PERIODIC && L > k.bigL) {
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
        const bool open = act && !far && (guard || crit);
        if (act && !open) {
            if (!far) {
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
                if (PERIODIC && L > k.bigL) {
                    qx = wrap_min_image(qx, k);
                    qy = wrap_min_image(qy, k);
                    qz = wrap_min_image(qz, k);
                }
                const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                if (!TREEPM || q2 <= k.rcut2) {
                    pair_term<TREEPM>(qx, qy, qz, q2, P.w, k, ax, ay, az, ph);
                    cnt++;
                }
            }
        }
        n = Lk.x;
    }
    if (!valid)
        return;
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

template <bool P, bool R, bool T>
void launch(const System *s, const WalkRequest &r, const WalkConsts &k, cudaStream_t st) {
    const int64_t warps = (r.n_act + 31) / 32;
    const int64_t blocks = (warps * 32 + kWalkThreads - 1) / kWalkThreads;
    k_walk<P, R, T><<<(unsigned)blocks, kWalkThreads, 0, st>>>(
        s->ncen, s->ncom, s->nlink, s->spart, s->key, s->perm, s->pos, s->x0[0], s->x0[1], s->x0[2], s->L0,
        (int)s->nnodes, r.sorted_idx, r.slot, r.a_old, r.n_act, k, r.acc, r.pot, r.nint, r.accumulate);
    count_launch();
}

}  // namespace

int walk_device(Ctx *, const System *s, const tpm_force_params *p, const WalkRequest &r, cudaStream_t st) {
    if (r.n_act == 0)
        return TPM_OK;
    WalkConsts k{};
    const double h = s->bp.h;
    k.h2 = (float)(h * h);
    k.hinv = (float)(1.0 / h);
    k.hinv3 = (float)(1.0 / (h * h * h));
    k.thr_const = (float)(p->theta * p->theta);
    k.alpha_over_G = (float)(p->alpha / s->bp.G);
    k.G = (float)s->bp.G;
    k.box_guard = p->box_guard ? 1 : 0;
    k.box = (float)s->bp.box;
    k.boxinv = (float)(1.0 / s->bp.box);
    k.bigL = (float)(0.25 * s->bp.box);
    if (p->treepm) {
        const double rs = p->asmth * s->bp.box / p->pm_n;
        const double rc = p->rcut * rs;
        k.rcut2 = (float)(rc * rc);
        k.inv2rs = (float)(1.0 / (2.0 * rs));
    }
    const bool per = s->bp.periodic != 0, rel = p->crit == TPM_CRIT_RELATIVE, tpm = p->treepm != 0;
    if (!per && !rel && !tpm)
        launch<false, false, false>(s, r, k, st);
    else if (!per && rel && !tpm)
        launch<false, true, false>(s, r, k, st);
    else if (per && !rel && tpm)
        launch<true, false, true>(s, r, k, st);
    else if (per && rel && tpm)
        launch<true, true, true>(s, r, k, st);
    else {
        set_error("unsupported walk mode (periodic systems need treepm = 1, open systems treepm = 0)");
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
