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
//   --  complex-to-real FFT -> the potential mesh (64 MiB at 256^3: it stays
//       in the 129 MB L2 for the interpolation)
//   K8  per active particle: the 4-point finite difference
//       dPhi/dx ~ [2/3 (Phi_{+1} - Phi_{-1}) - 1/12 (Phi_{+2} - Phi_{-2})] / dx
//       at each of the 8 CIC mesh points around the particle (circular on the
//       mesh), CIC-interpolated, and the CIC-interpolated potential.  The
//       difference is a circular convolution, so forming it in k-space (its
//       transfer function i [4/3 sin(theta) - 1/6 sin(2 theta)] / dx) would
//       give the same force meshes; differencing the one potential mesh here
//       saves three inverse transforms and four mesh passes, at the price of
//       FP32 cancellation in differences of a smooth potential (a relative
//       error near 1e-5 of the mesh force at the box scale, far below the
//       method's own).
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
// of the periodic Green's function and keeps k = 0; K8 differences the padded
// potential mesh circularly, like the periodic one.
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

// CIC mass assignment (Sec. 3.3) onto the periodic ng^3 mesh: each particle,
// taken in key order, adds its mass with trilinear weights to the 8 mesh
// points around it (mesh points at i / cells_per_len, wrapped), one float
// atomic per point.
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

// Per-axis factors of the Green's functions for mesh index i of an m-point
// axis (frequency n = i or i - m): tab[i] = (kfund n)^2 and tab[m + i] =
// sinc^2(theta / 2) with theta = 2 pi n / m (the CIC window of one axis).
__device__ __forceinline__ void green_axis_table(float *tab, int m, float kfund) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int n = i < m / 2 ? i : i - m;
        const float ka = kfund * (float)n;
        tab[i] = ka * ka;
        const float sc = sinc_f((float)kPi * (float)n / (float)m);
        tab[m + i] = sc * sc;
    }
    __syncthreads();
}

constexpr int kGreenThreads = 256;

// K7 on the r2c half spectrum [ng][ng][ng/2+1], in place: the potential
// spectrum.  A warp takes whole rows (ix, iy) and walks iz, so no index needs
// a division; the per-axis factors come from a table in shared memory, filled
// once per block.
__global__ void __launch_bounds__(kGreenThreads)
    k_green(cufftComplex *__restrict__ spec, int ng, float kfund, float rs2, float pref) {
    extern __shared__ float tab[];
    green_axis_table(tab, ng, kfund);
    const int nzh = ng / 2 + 1;
    const int64_t rows = (int64_t)ng * ng;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const int ix = (int)(r / ng), iy = (int)(r - (int64_t)ix * ng);
        const float kxy = tab[ix] + tab[iy], wxy = tab[ng + ix] * tab[ng + iy];
        cufftComplex *__restrict__ row = spec + r * nzh;
        for (int iz = lane; iz < nzh; iz += 32) {
            const float k2 = kxy + tab[iz];
            const float w2 = wxy * tab[ng + iz];  // W(k) = prod_a sinc^2(k_a dx / 2)
            float g = 0.0f;
            if (k2 > 0.0f)
                g = pref * __expf(-k2 * rs2) / (k2 * w2 * w2);
            const cufftComplex v = row[iz];
            row[iz] = make_float2(v.x * g, v.y * g);
        }
    }
}

// The spectral mesh force of one axis: out = -i k_a Phi_k on the half
// spectrum [ng][ng][ng/2+1] (Phi_k already carries the Green's function and
// the inverse transform's 1/ng^3); the Nyquist mode of the axis, whose
// derivative a real mesh cannot carry, gets zero.
__global__ void __launch_bounds__(kGreenThreads)
    k_spec_grad(const cufftComplex *__restrict__ spec, cufftComplex *__restrict__ out, int ng, int axis,
                float kfund) {
    const int nzh = ng / 2 + 1;
    const int64_t rows = (int64_t)ng * ng;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const int ix = (int)(r / ng), iy = (int)(r - (int64_t)ix * ng);
        const int nx = ix < ng / 2 ? ix : ix - ng, ny = iy < ng / 2 ? iy : iy - ng;
        const cufftComplex *__restrict__ row = spec + r * nzh;
        cufftComplex *__restrict__ orow = out + r * nzh;
        for (int iz = lane; iz < nzh; iz += 32) {
            const int n = axis == 0 ? nx : axis == 1 ? ny : iz;
            const float k = (2 * n == ng || 2 * n == -ng) ? 0.0f : kfund * (float)n;
            const cufftComplex v = row[iz];
            orow[iz] = make_float2(k * v.y, -k * v.x);  // -i k (re + i im)
        }
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

// Real parts of a complex array (the transform of the real, even isolated
// kernel).
__global__ void k_real_part(const cufftComplex *__restrict__ spec, int64_t nspec, float *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nspec;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = spec[e].x;  // the kernel is real and even: its transform is real
}

// K7 for open boundaries on the padded half spectrum [n2][n2][n2/2+1], in
// place: Phi_k = m_k g_k / W(k)^2 (pref = G / dx / n2^3 scales the mesh-unit
// kernel transform and folds in the inverse-FFT normalisation); rows as in
// k_green.
__global__ void __launch_bounds__(kGreenThreads)
    k_green_iso(cufftComplex *__restrict__ spec, int n2, const float *__restrict__ gk, float pref) {
    extern __shared__ float tab[];
    green_axis_table(tab, n2, 0.0f);
    const int nzh = n2 / 2 + 1;
    const int64_t rows = (int64_t)n2 * n2;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const int ix = (int)(r / n2), iy = (int)(r - (int64_t)ix * n2);
        const float wxy = tab[n2 + ix] * tab[n2 + iy];
        cufftComplex *__restrict__ row = spec + r * nzh;
        const float *__restrict__ grow = gk + r * nzh;
        for (int iz = lane; iz < nzh; iz += 32) {
            const float w2 = wxy * tab[n2 + iz];
            const float g = pref * grow[iz] / (w2 * w2);
            const cufftComplex v = row[iz];
            row[iz] = make_float2(v.x * g, v.y * g);
        }
    }
}

__device__ __forceinline__ int wrapi(int i, int ng) {
    i %= ng;
    return i < 0 ? i + ng : i;
}

// K8 core: potential and force at a particle whose CIC cell starts at mesh
// point i0 with fractions f, from the m^3 potential mesh, indices circular.
// The force at each of the 8 CIC points is minus the 4-point difference of
// the potential along each axis.  The six mesh values of a line along an axis
// through two neighbouring CIC points give both points' differences; the 8
// CIC points' own values come from the x lines and are kept for the y and z
// lines (56 loads, all within 3 cells of the particle).
__device__ __forceinline__ void pm_interp_point(const float *__restrict__ phi, int m, const int i0[3],
                                                const float f[3], float inv_dx, float &ph, float &gx, float &gy,
                                                float &gz) {
    int x[6], y[6], z[6];  // circular indices i0 - 2 .. i0 + 3 per axis
#pragma unroll
    for (int t = 0; t < 6; t++) {
        x[t] = wrapi(i0[0] - 2 + t, m);
        y[t] = wrapi(i0[1] - 2 + t, m);
        z[t] = wrapi(i0[2] - 2 + t, m);
    }
    const float wx[2] = {1.0f - f[0], f[0]}, wy[2] = {1.0f - f[1], f[1]}, wz[2] = {1.0f - f[2], f[2]};
    const float c1 = 2.0f / 3.0f * inv_dx, c2 = 1.0f / 12.0f * inv_dx;
    auto at = [&](int a, int b, int c) { return __ldg(&phi[((size_t)a * m + b) * m + c]); };
    float core[2][2][2];  // the CIC points' potentials [dx][dy][dz]
    ph = gx = gy = gz = 0.0f;
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {  // x line through (y[2 + u], z[2 + v])
            float l[6];
#pragma unroll
            for (int t = 0; t < 6; t++)
                l[t] = at(x[t], y[2 + u], z[2 + v]);
#pragma unroll
            for (int d = 0; d < 2; d++) {
                core[d][u][v] = l[2 + d];
                const float w = wx[d] * wy[u] * wz[v];
                ph = fmaf(w, l[2 + d], ph);
                gx = fmaf(w, c2 * (l[4 + d] - l[d]) - c1 * (l[3 + d] - l[1 + d]), gx);
            }
        }
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
            {  // y line through (x[2 + u], z[2 + v])
                const float l[6] = {at(x[2 + u], y[0], z[2 + v]), at(x[2 + u], y[1], z[2 + v]), core[u][0][v],
                                    core[u][1][v], at(x[2 + u], y[4], z[2 + v]), at(x[2 + u], y[5], z[2 + v])};
#pragma unroll
                for (int d = 0; d < 2; d++)
                    gy = fmaf(wx[u] * wy[d] * wz[v], c2 * (l[4 + d] - l[d]) - c1 * (l[3 + d] - l[1 + d]), gy);
            }
            {  // z line through (x[2 + u], y[2 + v])
                const float l[6] = {at(x[2 + u], y[2 + v], z[0]), at(x[2 + u], y[2 + v], z[1]), core[u][v][0],
                                    core[u][v][1], at(x[2 + u], y[2 + v], z[4]), at(x[2 + u], y[2 + v], z[5])};
#pragma unroll
                for (int d = 0; d < 2; d++)
                    gz = fmaf(wx[u] * wy[v] * wz[d], c2 * (l[4 + d] - l[d]) - c1 * (l[3 + d] - l[1 + d]), gz);
            }
        }
}

// K8 for open boundaries: from the padded potential mesh.  (Gather-bound:
// 64 registers admit four blocks per SM, 213 vs 223 us at 72 on the 256^3
// box.)
__global__ void __launch_bounds__(kThreads, 4) k_pm_interp_iso(const float *__restrict__ phi, int n2, double cx, double cy, double cz,
                                double cells_per_len, float inv_dx, const double *__restrict__ pos,
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
    float ph, gx, gy, gz;
    pm_interp_point(phi, n2, i0, f, inv_dx, ph, gx, gy, gz);
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

// K8: from the periodic potential mesh.
__global__ void __launch_bounds__(kThreads, 4) k_pm_interp(const float *__restrict__ phi, int ng, double cells_per_len, float inv_dx,
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
    float ph, gx, gy, gz;
    pm_interp_point(phi, ng, i0, f, inv_dx, ph, gx, gy, gz);
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

// K8 with the spectral force meshes (periodic): CIC interpolation of the
// three force meshes and the potential mesh, 32 loads per particle.
__global__ void __launch_bounds__(kThreads, 4)
    k_pm_interp_meshes(const float *__restrict__ phi, const float *__restrict__ fm, int ng, double cells_per_len,
                       const double *__restrict__ pos, const uint32_t *__restrict__ perm,
                       const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot, int64_t n_act,
                       float *__restrict__ acc, float *__restrict__ pot) {
    int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= n_act)
        return;
    const uint32_t s = sidx ? sidx[gi] : (uint32_t)gi;
    const uint32_t out = slot ? slot[gi] : perm[s];
    const uint32_t j = perm[s];
    int i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = pos[3 * j + a] * cells_per_len;
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        i0[a] = wrapi((int)fl, ng);
        i1[a] = wrapi(i0[a] + 1, ng);
    }
    const size_t cell = (size_t)ng * ng * ng;
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int ix = (c & 4) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 1) ? i1[2] : i0[2];
        const float w = ((c & 4) ? f[0] : 1.0f - f[0]) * ((c & 2) ? f[1] : 1.0f - f[1]) *
                        ((c & 1) ? f[2] : 1.0f - f[2]);
        const size_t q = ((size_t)ix * ng + iy) * ng + iz;
        ph = fmaf(w, __ldg(&phi[q]), ph);
        gx = fmaf(w, __ldg(&fm[q]), gx);
        gy = fmaf(w, __ldg(&fm[cell + q]), gy);
        gz = fmaf(w, __ldg(&fm[2 * cell + q]), gz);
    }
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

// cuFFT plans for an m^3 mesh (R2C and C2R), cached.
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
    if (cufftPlan3d(inv, m, m, m, CUFFT_C2R) != CUFFT_SUCCESS) {
        cufftDestroy(*fwd);
        set_error("cufftPlan3d (C2R, %d^3) failed", m);
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
        TPM_CHECK(s->pm_mem.get(&s->phi, ncell, st));
        s->pm_mesh = n2;
    }
    s->pm_n = ng;
    s->pm_grad = TPM_GRAD_FD4;
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
    TPM_CHECK(tmp.get(&spec, nspec, st));
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
    k_green_iso<<<(unsigned)(c->num_sms * 8), kGreenThreads, 2 * n2 * sizeof(float), st>>>(spec, n2, gk,
                                                                                              (float)pref);
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
    const bool ik = p->pm_grad == TPM_GRAD_IK;
    if (s->pm_mesh != ng || (ik && !s->fmesh)) {
        s->pm_mem.release(st);
        s->phi = nullptr;
        s->fmesh = nullptr;
        s->pm_mem.ctx = c;
        TPM_CHECK(s->pm_mem.get(&s->phi, ncell, st));
        if (ik)
            TPM_CHECK(s->pm_mem.get(&s->fmesh, 3 * ncell, st));
        s->pm_mesh = ng;
    }
    s->pm_n = ng;
    s->pm_grad = p->pm_grad;
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    cufftComplex *spec;
    TPM_CHECK(tmp.get(&spec, nspec, st));
    float *rho = s->phi;  // the density occupies the potential mesh until the inverse FFT
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
    k_green<<<(unsigned)(c->num_sms * 8), kGreenThreads, 2 * ng * sizeof(float), st>>>(
        spec, ng, (float)(2.0 * kPi / box), (float)(rs * rs), (float)pref);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(inv, st) != CUFFT_SUCCESS) {
        set_error("cufftSetStream failed");
        return TPM_ECUDA;
    }
    if (ik) {  // the force spectra first: the inverse transform may overwrite its input
        cufftComplex *gspec;
        TPM_CHECK(tmp.get(&gspec, nspec, st));
        for (int a = 0; a < 3; a++) {
            k_spec_grad<<<(unsigned)(c->num_sms * 8), kGreenThreads, 0, st>>>(spec, gspec, ng, a,
                                                                              (float)(2.0 * kPi / box));
            count_launch();
            TPM_CUDA(cudaGetLastError());
            if (cufftExecC2R(inv, gspec, s->fmesh + a * ncell) != CUFFT_SUCCESS) {
                set_error("cufftExecC2R (force mesh) failed");
                return TPM_ECUDA;
            }
        }
    }
    if (cufftExecC2R(inv, spec, s->phi) != CUFFT_SUCCESS) {
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
            s->phi, n2, s->pm_corner[0], s->pm_corner[1], s->pm_corner[2], s->pm_n / s->L0,
            (float)(s->pm_n / s->L0), s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        return TPM_OK;
    }
    const int ng = s->pm_n;
    const double box = s->bp.box;
    if (s->pm_grad == TPM_GRAD_IK) {
        k_pm_interp_meshes<<<(unsigned)((r.n_act + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            s->phi, s->fmesh, ng, ng / box, s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        return TPM_OK;
    }
    k_pm_interp<<<(unsigned)((r.n_act + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        s->phi, ng, ng / box, (float)(ng / box), s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
