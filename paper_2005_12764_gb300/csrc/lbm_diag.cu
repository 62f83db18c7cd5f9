// lbm_diag.cu -- diagnostics of the colour field, off the time step: the droplet
// census of the dense emulsion and the structure factor of the bicontinuous gel.
//
// Droplet census: the connected components of {phi > 0} under 26-connectivity
// (face, edge and corner neighbours), wrapping around periodic axes and not across
// walls. A lock-free union-find over node indices: every positive node starts as its
// own root; for each of 13 neighbour offsets (one of every opposite pair) the two
// roots are joined by pointing the larger at the smaller with atomicMin; roots only
// ever point to smaller indices, so every find walks a strictly decreasing chain.
// Then labels are flattened, component sizes counted and the roots' sizes listed.
//
// Structure factor: the radially averaged power spectrum of phi - mean(phi),
// S(k_b) = sum over modes in shell b of |phi_hat|^2 / (N * modes in shell b), shell
// b = round(|k| / dk), dk = 2 pi / max(n), from a single-precision real-to-complex
// FFT (cuFFT, a library call on a diagnostic path) and a shell sum in FP64.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_ctx.cuh"

namespace {

constexpr int kT = 256;

int blocks_for(size_t n, int num_sms) {
    size_t b = (n + kT - 1) / kT;
    const size_t cap = (size_t)num_sms * 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

__global__ void cc_init(const float* phi, size_t N, int* parent, int* size) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        parent[n] = phi[n] > 0.0f ? (int)n : -1;
        size[n] = 0;
    }
}

// Root of x. Parents only decrease, so the walk is at most x steps; the loads go
// through L2 (other threads link roots meanwhile).
__device__ __forceinline__ int cc_find(int* parent, int x) {
    int p = __ldcg(parent + x);
    while (p != x) {
        x = p;
        p = __ldcg(parent + x);
    }
    return x;
}

// Joins the components of a and b. Each retry starts from a smaller index, so the
// loop ends within a steps; the bound is a guard that records a failure instead.
__device__ __forceinline__ void cc_unite(int* parent, int a, int b, int* err) {
    for (int it = 0; it < (1 << 30); ++it) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    atomicExch(err, 1);
}

__global__ void cc_union(const StepParams p, int* parent, int* err) {
    const size_t N = p.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        if (__ldcg(parent + n) < 0) continue;
        const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny);
        const int z = (int)(n / ((size_t)p.nx * p.ny));
        for (int k = 14; k < 27; ++k) {   // offsets (dz, dy, dx) > (0, 0, 0)
            const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
            int xs = x + dx, ys = y + dy, zs = z + dz;
            xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
            if (ys < 0 || ys >= p.ny) {
                if (p.wall_y) continue;
                ys = ys < 0 ? ys + p.ny : ys - p.ny;
            }
            if (zs < 0 || zs >= p.nz) {
                if (p.wall_z) continue;
                zs = zs < 0 ? zs + p.nz : zs - p.nz;
            }
            const size_t m = ((size_t)zs * p.ny + ys) * p.nx + xs;
            if (__ldcg(parent + m) < 0) continue;
            cc_unite(parent, (int)n, (int)m, err);
        }
    }
}

__global__ void cc_count(size_t N, int* parent, int* size) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        if (parent[n] < 0) continue;
        atomicAdd(size + cc_find(parent, (int)n), 1);
    }
}

__global__ void cc_collect(size_t N, const int* size, int* out, int* count) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int s = size[n];
        if (s > 0) out[atomicAdd(count, 1)] = s;
    }
}

__global__ void sum_kernel(const float* v, size_t N, double* out) {
    double a = 0.0;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x)
        a += v[n];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, a);
}

__global__ void centre_kernel(const float* v, size_t N, const double* sum, float* out) {
    const float mean = (float)(*sum / (double)N);
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x)
        out[n] = v[n] - mean;
}

// Shell sums over the half spectrum [nz][ny][nx/2 + 1]: modes m_x = 0 (and n_x/2 for
// even n_x) stand for themselves, the others also for their conjugates (-m_x). The
// shell index is computed in FP64 with explicit roundings, as round(2 pi |m/n| / dk).
__global__ void shell_kernel(const cufftComplex* F, int nx, int ny, int nz, int nbins, double dk,
                             double* S, unsigned long long* cnt) {
    const int hx = nx / 2 + 1;
    const size_t M = (size_t)nz * ny * hx;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < M;
         q += (size_t)gridDim.x * blockDim.x) {
        const int mx = (int)(q % hx);
        const int iy = (int)((q / hx) % ny), iz = (int)(q / ((size_t)hx * ny));
        const int my = iy < (ny + 1) / 2 ? iy : iy - ny;   // fftfreq order
        const int mz = iz < (nz + 1) / 2 ? iz : iz - nz;
        const double ax = __ddiv_rn((double)mx, (double)nx);
        const double ay = __ddiv_rn((double)my, (double)ny);
        const double az = __ddiv_rn((double)mz, (double)nz);
        const double k2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
        const double kk = __dmul_rn(2.0 * 3.141592653589793, __dsqrt_rn(k2));
        const double bf = rint(__ddiv_rn(kk, dk));
        if (!(bf < (double)nbins)) continue;
        const int b = (int)bf;
        const int w = (mx == 0 || (nx % 2 == 0 && mx == nx / 2)) ? 1 : 2;
        const double re = F[q].x, im = F[q].y;
        atomicAdd(S + b, (double)w * (re * re + im * im));
        atomicAdd(cnt + b, (unsigned long long)w);
    }
}

}  // namespace

using namespace lbm;

extern "C" lbm_status lbm_droplets(lbm_ctx* c, long long* count, long long* sizes,
                                   long long capacity) {
    if (!c || !count) return LBM_EINVAL;
    if (!c->fields_set) return ctx_fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    if (capacity < 0 || (capacity > 0 && !sizes)) return ctx_fail(c, LBM_EINVAL, "sizes/capacity");
    const size_t N = c->N;
    if (N >= (size_t)1 << 31) return ctx_fail(c, LBM_EINVAL, "more than 2^31 - 1 nodes");
    // parent [N] and size [N] ints in the staging buffer, plus the error word and count
    if (ctx_stage(c, N + 2) != LBM_OK) return LBM_ENOMEM;
    int* parent = reinterpret_cast<int*>(c->stage);
    int* size = parent + N;
    int* word = size + N;   // [0] error, [1] component count
    cudaStream_t s = c->stream;
    const int grid = blocks_for(N, c->num_sms);
    cudaError_t e = cudaMemsetAsync(word, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) {
        cc_init<<<grid, kT, 0, s>>>(c->phi[c->pc], N, parent, size);
        cc_union<<<grid, kT, 0, s>>>(c->sp, parent, word);
        cc_count<<<grid, kT, 0, s>>>(N, parent, size);
        cc_collect<<<grid, kT, 0, s>>>(N, size, parent, word + 1);   // parent reused
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, word, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return ctx_fail(c, LBM_ECUDA, std::string("droplet census: ") + cudaGetErrorString(e));
    if (h[0]) return ctx_fail(c, LBM_ECUDA, "droplet census: a union did not settle");
    *count = h[1];
    if (capacity > 0 && h[1] > 0) {
        std::vector<int> v((size_t)h[1]);
        e = cudaMemcpy(v.data(), parent, v.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return ctx_fail(c, LBM_ECUDA, std::string("droplet census: ") + cudaGetErrorString(e));
        std::sort(v.begin(), v.end(), [](int a, int b) { return a > b; });
        const size_t k = std::min((size_t)capacity, v.size());
        for (size_t i = 0; i < k; ++i) sizes[i] = v[i];
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_structure_factor(lbm_ctx* c, int nbins, double* k, double* S,
                                           long long* modes) {
    if (!c || nbins < 1 || !S) return LBM_EINVAL;
    if (!c->fields_set) return ctx_fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    const size_t N = c->N;
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const size_t half = (size_t)nz * ny * (nx / 2 + 1);
    // staging: the centred field (N floats), the half spectrum (2 floats per mode) and
    // the shell sums, in doubles
    const size_t dbl = (N + 1) / 2 + half + 1 + 2 * (size_t)nbins + 1;
    if (ctx_stage(c, dbl) != LBM_OK) return LBM_ENOMEM;
    float* centred = reinterpret_cast<float*>(c->stage);
    cufftComplex* F = reinterpret_cast<cufftComplex*>(c->stage + (N + 1) / 2);
    double* sum = c->stage + (N + 1) / 2 + half;
    double* dS = sum + 1;
    unsigned long long* dcnt = reinterpret_cast<unsigned long long*>(dS + nbins);
    cudaStream_t s = c->stream;
    const int grid = blocks_for(N, c->num_sms);
    cudaError_t e = cudaMemsetAsync(sum, 0, (1 + 2 * (size_t)nbins) * sizeof(double), s);
    if (e == cudaSuccess) {
        sum_kernel<<<grid, kT, 0, s>>>(c->phi[c->pc], N, sum);
        centre_kernel<<<grid, kT, 0, s>>>(c->phi[c->pc], N, sum, centred);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return ctx_fail(c, LBM_ECUDA, std::string("structure factor: ") + cudaGetErrorString(e));
    cufftHandle plan;
    if (cufftPlan3d(&plan, nz, ny, nx, CUFFT_R2C) != CUFFT_SUCCESS)
        return ctx_fail(c, LBM_ENOMEM, "structure factor: FFT plan");
    cufftResult r = cufftSetStream(plan, s);
    if (r == CUFFT_SUCCESS) r = cufftExecR2C(plan, centred, F);
    if (r != CUFFT_SUCCESS) {
        cufftDestroy(plan);
        return ctx_fail(c, LBM_ECUDA, "structure factor: FFT");
    }
    const double dk = 2.0 * 3.141592653589793 / (double)std::max(nx, std::max(ny, nz));
    shell_kernel<<<blocks_for(half, c->num_sms), kT, 0, s>>>(F, nx, ny, nz, nbins, dk, dS, dcnt);
    e = cudaGetLastError();
    std::vector<double> hS((size_t)nbins);
    std::vector<unsigned long long> hc((size_t)nbins);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hS.data(), dS, nbins * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hc.data(), dcnt, nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cufftDestroy(plan);
    if (e != cudaSuccess)
        return ctx_fail(c, LBM_ECUDA, std::string("structure factor: ") + cudaGetErrorString(e));
    for (int b = 0; b < nbins; ++b) {
        S[b] = hc[b] ? hS[b] / ((double)N * (double)hc[b]) : 0.0;
        if (k) k[b] = dk * b;
        if (modes) modes[b] = (long long)hc[b];
    }
    return LBM_OK;
}
