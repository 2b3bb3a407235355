// Periodic particle-mesh long-range force (paper Sec. 3.3, 3.4).
//
//   K6  cloud-in-cell assignment of every particle's mass to the 8 mesh points
//       around it (mesh points at x = i box / N), FP32 atomics
//   --  real-to-complex FFT (cuFFT)
//   K7  multiply by the Green's function of the long-range potential,
//       -4 pi G / k^2 exp(-k^2 r_s^2), divided by the square of the CIC window
//       W(k) = prod_a sinc^2(k_a dx / 2) (one window for assignment, one for
//       interpolation), with the k = 0 mode removed (the mean density does not
//       source the potential) and the inverse-FFT normalisation folded in.
//       The same pass also forms the three force spectra: the 4-point
//       finite difference dPhi/dx ~ [4/3 (Phi_{+1} - Phi_{-1})/2 -
//       1/3 (Phi_{+2} - Phi_{-2})/4] / dx is a circular convolution on the
//       periodic mesh, so it equals multiplication by its transfer function
//       i [4/3 sin(theta) - 1/6 sin(2 theta)] / dx, theta = 2 pi n / N.
//       Applying it in k-space gives the finite-difference force mesh without
//       the FP32 cancellation of differencing a smooth potential.
//   --  one batched complex-to-real FFT -> potential and 3 force meshes
//   K8  per active particle: CIC interpolation of force and potential
//
// Open boundaries (Sec. 3.3: zero padding and the Green's function of
// isolated boundaries).  The mesh covers a cube of the tree root's side
// centred on the particles (at least a tenth of the side free on every side)
// with pm_n points per side, inside a zero-padded (2 pm_n)^3 mesh.  The
// potential is the convolution of the CIC masses with the long-range kernel
// g(r) = -G erf(r / 2 r_s) / r, g(0) = -G / (sqrt(pi) r_s), sampled at the
// padded mesh's circular separations min(|i|, 2 pm_n - |i|) dx: the circular
// convolution equals the open one on the physical region.  The transform of
// the kernel (in mesh units, per padded size and split scale in cells) is
// computed once per context; K7 multiplies by it (scaled by G / dx) instead
// of the periodic Green's function, keeps k = 0, and forms the same
// finite-difference force spectra on the padded mesh, which equal the
// real-space differences wherever the stencil stays inside the physical
// region.
#include <map>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kThreads = 256;
constexpr double kPi = 3.14159265358979323846;

// Adds v to rho[idx] with one atomic per distinct address in the warp: lanes
// that target the same mesh point (common for key-ordered particles, and
// dominant in the dense centre of a halo) sum their contributions first.
// Every lane of the warp must call this; a lane with idx == UINT32_MAX adds
// nothing (meshes have at most 2^30 points).
__device__ __forceinline__ void warp_add(float *__restrict__ rho, unsigned idx, float v) {
    const unsigned peers = __match_any_sync(0xffffffffu, idx);
    float sum = 0.0f;
    for (unsigned todo = peers; todo; todo &= todo - 1)
        sum += __shfl_sync(peers, v, __ffs(todo) - 1);
    if ((threadIdx.x & 31) == __ffs(peers) - 1 && idx != ~0u)
        atomicAdd(&rho[idx], sum);
}

__global__ void k_cic_deposit(const double *__restrict__ pos, const float *__restrict__ mass,
                              const uint32_t *__restrict__ perm, int64_t n, int ng, double cells_per_len,
                              float *__restrict__ rho) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = s < n;
    const uint32_t j = live ? perm[s] : 0u;  // key order: neighbouring threads hit neighbouring cells
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = pos[3 * j + a] * cells_per_len;
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        int q = (int)fl;
        q %= ng;
        if (q < 0)
            q += ng;
        i0[a] = q;
    }
    const float m = live ? mass[j] : 0.0f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
        ix -= ix >= ng ? ng : 0;
        iy -= iy >= ng ? ng : 0;
        iz -= iz >= ng ? ng : 0;
        // a periodic box is close to uniform on the mesh scale: plain atomics
        // (the warp aggregation of the open-boundary deposit costs more here)
        if (live)
            atomicAdd(&rho[((size_t)ix * ng + iy) * ng + iz], m * w);
    }
}

// sin(x)/x with the accurate sinf: the fast __sinf has an absolute error of
// ~4e-7, i.e. a relative error of ~3e-5 at the fundamental mode of a 256^3 mesh.
__device__ __forceinline__ float sinc_f(float x) { return x == 0.0f ? 1.0f : sinf(x) / x; }

// K7 on the r2c half spectrum [ng][ng][ng/2+1]: spec[0] (in place) becomes the
// potential spectrum, spec[1..3] the x, y, z force spectra.
__global__ void k_green(cufftComplex *__restrict__ spec, int64_t nspec, int ng, float kfund, float dx, float rs2,
                        float pref) {
    const int nzh = ng / 2 + 1;
    const float inv_dx = 1.0f / dx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nspec;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % nzh);
        const int iy = (int)((e / nzh) % ng);
        const int ix = (int)(e / ((int64_t)nzh * ng));
        const int n3[3] = {ix < ng / 2 ? ix : ix - ng, iy < ng / 2 ? iy : iy - ng, iz};
        float k2 = 0.0f, w = 1.0f, d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float ka = kfund * n3[a];
            k2 = fmaf(ka, ka, k2);
            w *= sinc_f(0.5f * ka * dx);
            const float th = 2.0f * (float)n3[a] / (float)ng;  // theta / pi
            d[a] = (4.0f / 3.0f * sinpif(th) - 1.0f / 6.0f * sinpif(2.0f * th)) * inv_dx;
        }
        cufftComplex v = spec[e];
        float g = 0.0f;
        if (k2 > 0.0f) {
            const float w2 = w * w;  // sinc^2 per axis
            g = pref * __expf(-k2 * rs2) / (k2 * w2 * w2);
        }
        const float re = v.x * g, im = v.y * g;
        spec[e] = make_float2(re, im);
        // force = -grad Phi: multiply by -i d
#pragma unroll
        for (int a = 0; a < 3; a++)
            spec[(a + 1) * nspec + e] = make_float2(d[a] * im, -d[a] * re);
    }
}

// Open boundaries: CIC masses (not densities) into the corner ng^3 block of
// the zero-padded n2^3 mesh; mesh point i sits at corner + i / cells_per_len.
// Positions lie inside the block with a margin (no wrap needed).
__global__ void k_cic_deposit_iso(const double *__restrict__ pos, const float *__restrict__ mass,
                                  const uint32_t *__restrict__ perm, int64_t n, int n2, double cx, double cy,
                                  double cz, double cells_per_len, float *__restrict__ rho) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = s < n;  // dead lanes stay for the warp-wide aggregation
    const uint32_t j = live ? perm[s] : 0u;
    const double c0[3] = {cx, cy, cz};
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = __dmul_rn(__dsub_rn(pos[3 * j + a], c0[a]), cells_per_len);
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        i0[a] = min(max((int)fl, 0), n2 - 2);
    }
    const float m = live ? mass[j] : 0.0f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        warp_add(rho, live ? ((unsigned)(i0[0] + dx) * n2 + (i0[1] + dy)) * n2 + (i0[2] + dz) : ~0u, m * w);
    }
}

// The long-range kernel in mesh units (dx = 1, G = 1) on the padded mesh:
// -erf(r / 2 a_s) / r at the circular separation r, -1 / (sqrt(pi) a_s) at 0.
__global__ void k_iso_kernel(float *__restrict__ g, int n2, double asmth) {
    const int64_t total = (int64_t)n2 * n2 * n2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % n2), iy = (int)((e / n2) % n2), ix = (int)(e / ((int64_t)n2 * n2));
        const double dx = min(ix, n2 - ix), dy = min(iy, n2 - iy), dz = min(iz, n2 - iz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        g[e] = (float)(r > 0.0 ? -erf(r / (2.0 * asmth)) / r : -1.0 / (sqrt(kPi) * asmth));
    }
}

__global__ void k_real_part(const cufftComplex *__restrict__ spec, int64_t nspec, float *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nspec;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = spec[e].x;  // the kernel is real and even: its transform is real
}

// K7 for open boundaries on the padded half spectrum [n2][n2][n2/2+1]:
// Phi_k = m_k g_k / W(k)^2 (pref = G / dx / n2^3 scales the mesh-unit kernel
// transform and folds in the inverse-FFT normalisation), then the force
// spectra of the 4-point difference as in k_green.
__global__ void k_green_iso(cufftComplex *__restrict__ spec, int64_t nspec, int n2, const float *__restrict__ gk,
                            float dx, float pref) {
    const int nzh = n2 / 2 + 1;
    const float inv_dx = 1.0f / dx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nspec;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % nzh);
        const int iy = (int)((e / nzh) % n2);
        const int ix = (int)(e / ((int64_t)nzh * n2));
        const int n3[3] = {ix < n2 / 2 ? ix : ix - n2, iy < n2 / 2 ? iy : iy - n2, iz};
        float w = 1.0f, d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float th = 2.0f * (float)n3[a] / (float)n2;  // theta / pi
            w *= sinc_f(0.5f * (float)kPi * th);                // sinc(k_a dx / 2)
            d[a] = (4.0f / 3.0f * sinpif(th) - 1.0f / 6.0f * sinpif(2.0f * th)) * inv_dx;
        }
        const float w2 = w * w;
        const float g = pref * gk[e] / (w2 * w2);
        const cufftComplex v = spec[e];
        const float re = v.x * g, im = v.y * g;
        spec[e] = make_float2(re, im);
#pragma unroll
        for (int a = 0; a < 3; a++)
            spec[(a + 1) * nspec + e] = make_float2(d[a] * im, -d[a] * re);
    }
}

// K8 for open boundaries: CIC interpolation from the padded meshes.
__global__ void k_pm_interp_iso(const float *__restrict__ mesh, int64_t ncell, int n2, double cx, double cy,
                                double cz, double cells_per_len, const double *__restrict__ pos,
                                const uint32_t *__restrict__ perm, const uint32_t *__restrict__ sidx,
                                const uint32_t *__restrict__ slot, int64_t n_act, float *__restrict__ acc,
                                float *__restrict__ pot) {
    int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= n_act)
        return;
    const uint32_t s = sidx ? sidx[gi] : (uint32_t)gi;
    const uint32_t out = slot ? slot[gi] : perm[s];
    const uint32_t j = perm[s];
    const double c0[3] = {cx, cy, cz};
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = __dmul_rn(__dsub_rn(pos[3 * j + a], c0[a]), cells_per_len);
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        i0[a] = min(max((int)fl, 0), n2 - 2);
    }
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        const size_t idx = ((size_t)(i0[0] + dx) * n2 + (i0[1] + dy)) * n2 + (i0[2] + dz);
        ph = fmaf(w, __ldg(&mesh[idx]), ph);
        gx = fmaf(w, __ldg(&mesh[ncell + idx]), gx);
        gy = fmaf(w, __ldg(&mesh[2 * ncell + idx]), gy);
        gz = fmaf(w, __ldg(&mesh[3 * ncell + idx]), gz);
    }
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

__device__ __forceinline__ int wrapi(int i, int ng) {
    i %= ng;
    return i < 0 ? i + ng : i;
}

// K8: CIC interpolation of the force meshes and the potential mesh.
__global__ void k_pm_interp(const float *__restrict__ mesh, int64_t ncell, int ng, double cells_per_len,
                            const double *__restrict__ pos, const uint32_t *__restrict__ perm,
                            const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot, int64_t n_act,
                            float *__restrict__ acc, float *__restrict__ pot) {
    int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= n_act)
        return;
    const uint32_t s = sidx ? sidx[gi] : (uint32_t)gi;
    const uint32_t out = slot ? slot[gi] : perm[s];
    const uint32_t j = perm[s];
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = pos[3 * j + a] * cells_per_len;
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        i0[a] = wrapi((int)fl, ng);
    }
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        int x = i0[0] + dx, y = i0[1] + dy, z = i0[2] + dz;
        x -= x >= ng ? ng : 0;
        y -= y >= ng ? ng : 0;
        z -= z >= ng ? ng : 0;
        const size_t idx = ((size_t)x * ng + y) * ng + z;
        ph = fmaf(w, __ldg(&mesh[idx]), ph);
        gx = fmaf(w, __ldg(&mesh[ncell + idx]), gx);
        gy = fmaf(w, __ldg(&mesh[2 * ncell + idx]), gy);
        gz = fmaf(w, __ldg(&mesh[3 * ncell + idx]), gz);
    }
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

// cuFFT plans for an m^3 mesh (R2C, and C2R batched over four fields), cached.
int fft_plans_for(Ctx *c, int m, cufftHandle *fwd, cufftHandle *inv) {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->fft_plans.find(m);
    if (it != c->fft_plans.end()) {
        *fwd = it->second.first;
        *inv = it->second.second;
        return TPM_OK;
    }
    if (cufftPlan3d(fwd, m, m, m, CUFFT_R2C) != CUFFT_SUCCESS) {
        set_error("cufftPlan3d (R2C, %d^3) failed", m);
        return TPM_ECUDA;
    }
    int dims[3] = {m, m, m};
    if (cufftPlanMany(inv, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 4) != CUFFT_SUCCESS) {
        cufftDestroy(*fwd);
        set_error("cufftPlanMany (C2R x 4, %d^3) failed", m);
        return TPM_ECUDA;
    }
    c->fft_plans[m] = {*fwd, *inv};
    return TPM_OK;
}

// Transform of the isolated long-range kernel (mesh units) for an n2^3 padded
// mesh and split scale asmth cells: computed on first use, kept per context.
int iso_green_for(Ctx *c, int n2, double asmth, cufftHandle fwd, cudaStream_t st, const float **out) {
    const int64_t nspec = (int64_t)n2 * n2 * (n2 / 2 + 1);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->iso_green.find({n2, asmth});
        if (it != c->iso_green.end()) {
            *out = static_cast<const float *>(it->second.p);
            return TPM_OK;
        }
    }
    void *gk = nullptr;
    TPM_CHECK(ctx_alloc(c, &gk, nspec * sizeof(float), st));
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    float *g;
    cufftComplex *spec;
    int rc = tmp.get(&g, (size_t)n2 * n2 * n2, st);
    if (rc == TPM_OK)
        rc = tmp.get(&spec, nspec, st);
    if (rc != TPM_OK) {
        ctx_free(c, gk, nspec * sizeof(float), st);
        return rc;
    }
    k_iso_kernel<<<(unsigned)(c->num_sms * 8), kThreads, 0, st>>>(g, n2, asmth);
    count_launch();
    if (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftExecR2C(fwd, g, spec) != CUFFT_SUCCESS) {
        ctx_free(c, gk, nspec * sizeof(float), st);
        set_error("cufftExecR2C (isolated kernel) failed");
        return TPM_ECUDA;
    }
    k_real_part<<<(unsigned)(c->num_sms * 8), kThreads, 0, st>>>(spec, nspec, static_cast<float *>(gk));
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx_free(c, gk, nspec * sizeof(float), st);
        set_error("isolated kernel transform: %s", cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    c->iso_green[{n2, asmth}] = DevAlloc{gk, nspec * sizeof(float)};
    *out = static_cast<const float *>(gk);
    return TPM_OK;
}

int pm_solve_iso(Ctx *c, System *s, const tpm_force_params *p, cudaStream_t st) {
    const int ng = p->pm_n, n2 = 2 * ng;
    const double side = s->L0;
    const double dx = side / ng;
    const int64_t ncell = (int64_t)n2 * n2 * n2;
    const int64_t nspec = (int64_t)n2 * n2 * (n2 / 2 + 1);
    cufftHandle fwd, inv;
    TPM_CHECK(fft_plans_for(c, n2, &fwd, &inv));
    const float *gk;
    TPM_CHECK(iso_green_for(c, n2, p->asmth, fwd, st, &gk));
    if (s->pm_mesh != n2) {
        s->pm_mem.release(st);
        s->phi = nullptr;
        s->pm_mem.ctx = c;
        TPM_CHECK(s->pm_mem.get(&s->phi, 4 * ncell, st));
        s->pm_mesh = n2;
    }
    s->pm_n = ng;
    for (int a = 0; a < 3; a++)  // the region: a root-sized cube centred on the bounding box
        s->pm_corner[a] = (s->bb_lo[a] + s->bb_hi[a]) * 0.5 - 0.5 * side;
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    cufftComplex *spec;
    TPM_CHECK(tmp.get(&spec, 4 * nspec, st));
    float *rho = s->phi;
    TPM_CUDA(cudaMemsetAsync(rho, 0, ncell * sizeof(float), st));
    k_cic_deposit_iso<<<(unsigned)((s->n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        s->pos, s->mass, s->perm, s->n, n2, s->pm_corner[0], s->pm_corner[1], s->pm_corner[2], ng / side, rho);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftExecR2C(fwd, rho, spec) != CUFFT_SUCCESS) {
        set_error("cufftExecR2C failed");
        return TPM_ECUDA;
    }
    const double pref = s->bp.G / dx / (double)ncell;
    k_green_iso<<<(unsigned)(c->num_sms * 8), kThreads, 0, st>>>(spec, nspec, n2, gk, (float)dx, (float)pref);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(inv, st) != CUFFT_SUCCESS || cufftExecC2R(inv, spec, s->phi) != CUFFT_SUCCESS) {
        set_error("cufftExecC2R failed");
        return TPM_ECUDA;
    }
    s->pm_rs = p->asmth * dx;
    s->pm_G = s->bp.G;
    return TPM_OK;
}

}  // namespace

int pm_solve_device(Ctx *c, System *s, const tpm_force_params *p, cudaStream_t st) {
    if (!s->bp.periodic)
        return pm_solve_iso(c, s, p, st);
    const int ng = p->pm_n;
    const double box = s->bp.box;
    const double rs = p->asmth * box / ng;
    const int64_t ncell = (int64_t)ng * ng * ng;
    const int64_t nspec = (int64_t)ng * ng * (ng / 2 + 1);
    cufftHandle fwd, inv;
    TPM_CHECK(fft_plans_for(c, ng, &fwd, &inv));
    if (s->pm_mesh != ng) {
        s->pm_mem.release(st);
        s->phi = nullptr;
        s->pm_mem.ctx = c;
        TPM_CHECK(s->pm_mem.get(&s->phi, 4 * ncell, st));  // potential, then x, y, z force
        s->pm_mesh = ng;
    }
    s->pm_n = ng;
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    cufftComplex *spec;
    TPM_CHECK(tmp.get(&spec, 4 * nspec, st));
    float *rho = s->phi;  // the density occupies the potential slot until the inverse FFT
    TPM_CUDA(cudaMemsetAsync(rho, 0, ncell * sizeof(float), st));
    const double cpl = ng / box;
    k_cic_deposit<<<(unsigned)((s->n + kThreads - 1) / kThreads), kThreads, 0, st>>>(s->pos, s->mass, s->perm, s->n,
                                                                                     ng, cpl, rho);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftExecR2C(fwd, rho, spec) != CUFFT_SUCCESS) {
        set_error("cufftExecR2C failed");
        return TPM_ECUDA;
    }
    const double dx = box / ng;
    // density = mass / dx^3; inverse FFT normalisation 1 / ng^3
    const double pref = -4.0 * kPi * s->bp.G / (dx * dx * dx) / (double)ncell;
    k_green<<<(unsigned)(c->num_sms * 8), kThreads, 0, st>>>(spec, nspec, ng, (float)(2.0 * kPi / box), (float)dx,
                                                            (float)(rs * rs), (float)pref);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(inv, st) != CUFFT_SUCCESS || cufftExecC2R(inv, spec, s->phi) != CUFFT_SUCCESS) {
        set_error("cufftExecC2R failed");
        return TPM_ECUDA;
    }
    s->pm_rs = rs;
    s->pm_G = s->bp.G;
    return TPM_OK;
}

int pm_interp_device(Ctx *, const System *s, const WalkRequest &r, cudaStream_t st) {
    if (r.n_act == 0)
        return TPM_OK;
    if (!s->bp.periodic) {
        const int n2 = s->pm_mesh;
        k_pm_interp_iso<<<(unsigned)((r.n_act + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            s->phi, (int64_t)n2 * n2 * n2, n2, s->pm_corner[0], s->pm_corner[1], s->pm_corner[2], s->pm_n / s->L0,
            s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        return TPM_OK;
    }
    const int ng = s->pm_n;
    const double box = s->bp.box;
    k_pm_interp<<<(unsigned)((r.n_act + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        s->phi, (int64_t)ng * ng * ng, ng, ng / box, s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
