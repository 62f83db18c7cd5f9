// lbm_api.cu -- C-ABI of liblbm.so (declared in include/lbm.h): context and device
// memory management, field set/get conversions, FP64 reductions and the launch of
// the fused step kernel (lbm_step.cu).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbm.h"
#include "lbm_ctx.cuh"

using namespace lbm;

static thread_local std::string g_create_err;

namespace lbm {
// Error message of a failed call that has no context (read by lbm_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_err = msg; }
}  // namespace lbm

static lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c) c->err = msg; else g_create_err = msg;
    return s;
}
static lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(ctx, call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

// ---------------------------------------------------------------- aux kernels
namespace {

constexpr int kThreads = 256;

// Padded index of unpadded node n.
__device__ __forceinline__ size_t node_pidx(const StepParams& sp, size_t n) {
    const size_t plane = (size_t)sp.nx * sp.ny;
    const int z = (int)(n / plane);
    const int rem = (int)(n - (size_t)z * plane);
    const int y = rem / sp.nx, x = rem - y * sp.nx;
    return pidx(sp.pitch, sp.nyp, sp.padx, x, y, z);
}

// f_i^k = f_i^eq(rho_k, u), Eq. (2); both colour-field buffers get phi.
// Direction block a state write of f*_i of a node goes to, at the node's own padded
// index: i for the two-copy storage; opp(i) (layout 0) with in-place storage.
__device__ inline int wdir(const StepParams& sp, int i) { return sp.aa_layout < 0 ? i : opp(i); }
template <class St>
__global__ void init_fields_kernel(typename St::T* f, float* phi0, float* phi1,
                                   const double* rho_r, const double* rho_b, const double* u,
                                   StepParams sp) {
    // (node indices in 32 bits: a lattice has fewer than 2^31 nodes)
    const unsigned N = (unsigned)sp.N, plane = (unsigned)sp.nx * (unsigned)sp.ny;
    const size_t P = sp.P;
    const float ref_half = sp.ref_half;
    for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const unsigned z = n / plane, rem = n - z * plane;
        const unsigned y = rem / (unsigned)sp.nx, x = rem - y * (unsigned)sp.nx;
        const size_t q = pidx(sp.pitch, sp.nyp, sp.padx, (int)x, (int)y, (int)z);
        const double rr = rho_r[n], rb = rho_b[n];
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (u) {
            ux = (float)u[n];
            uy = (float)u[N + n];
            uz = (float)u[2 * (size_t)N + n];
        }
        const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
        const float ph = (float)((rr - rb) / (rr + rb));
        // f_i = rho_k w_i (1 + d_i), d_i = 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u^2: rho_k w_i per
        // weight class in FP64, rounded once, and the small correction d_i in FP32 (the
        // result within an FP32 unit of the FP64 value rounded)
        const float wr[3] = {(float)(rr * (1.0 / 3.0)), (float)(rr * (1.0 / 18.0)), (float)(rr * (1.0 / 36.0))};
        const float wb[3] = {(float)(rb * (1.0 / 3.0)), (float)(rb * (1.0 / 18.0)), (float)(rb * (1.0 / 36.0))};
        const double rho = rr + rb;
        const float wt[3] = {(float)(rho * (1.0 / 3.0)), (float)(rho * (1.0 / 18.0)), (float)(rho * (1.0 / 36.0))};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
            const float d = cu * (3.0f + 4.5f * cu) - usq15;
            const int c = csq(i);
            if constexpr (St::RED) {
                St::store(f, (size_t)i * P + q, __fmaf_rn(wt[c], d, wt[c]),
                          St::tot_ref(i, 2.0f * ref_half));
            } else {
                const float hw = wgt(i) * ref_half;
                const int dd = wdir(sp, i);
                St::store(f, (size_t)dd * P + q, __fmaf_rn(wr[c], d, wr[c]), dev_ref(hw, ph, 0));
                St::store(f, (size_t)(Q + dd) * P + q, __fmaf_rn(wb[c], d, wb[c]), dev_ref(hw, ph, 1));
            }
        }
        if constexpr (St::RED) {
            // f^eq is linear in the density: f^eq(rho_k, u) = (rho_k / rho) f^eq(rho, u),
            // the reduced form with kappa_k = rho_k / rho and m = 0
            St::store_coef(f, P, q, 0, (float)(rr / rho));
            St::store_coef(f, P, q, 1, (float)(rb / rho));
            for (int k = 2; k < Q5_AUX; ++k) St::store_coef(f, P, q, k, 0.0f);
        }
        phi0[n] = ph;
        phi1[n] = ph;
    }
}

// Population (species k, direction i) at padded index idx of a node whose current
// colour field is ph: deviation storage decodes against the reference of that node.
template <class St>
__device__ inline float ldpop(const typename St::T* f, size_t idx, int i, int k, float ref_half,
                              float ph) {
    return St::load(f, idx, dev_ref(wgt(i) * ref_half, ph, k));
}
// Both species' populations of direction i at padded index q (P = elements per
// block): stored as such, or in the reduced form rebuilt from the total and the
// node's recolouring coefficients.
template <class St>
__device__ inline void ldpair(const typename St::T* f, size_t P, size_t q, int i, float ref_half,
                              float ph, float& a, float& b) {
    if constexpr (St::RED) {
        const float t = St::load(f, (size_t)i * P + q, St::tot_ref(i, 2.0f * ref_half));
        const float sh = q5_share(i, St::coef(f, P, q, 2), St::coef(f, P, q, 3), St::coef(f, P, q, 4));
        a = __fmaf_rn(St::coef(f, P, q, 0), t, sh);
        b = __fmaf_rn(St::coef(f, P, q, 1), t, -sh);
    } else {
        a = ldpop<St>(f, (size_t)i * P + q, i, 0, ref_half, ph);
        b = ldpop<St>(f, (size_t)(Q + i) * P + q, i, 1, ref_half, ph);
    }
}
// Both species' populations f*_i of node n (padded index q) of the state: ldpair for
// the two-copy storage; with in-place storage from the slots the state's layout puts
// them in (aa_slot).
template <class St>
__device__ inline void ldnode(const typename St::T* f, const StepParams& sp, size_t n, size_t q,
                              int i, float ph, float& a, float& b) {
    if (sp.aa_layout < 0) {
        ldpair<St>(f, sp.P, q, i, sp.ref_half, ph, a, b);
        return;
    }
    const size_t plane = (size_t)sp.nx * sp.ny;
    const int z = (int)(n / plane);
    const int rem = (int)(n - (size_t)z * plane);
    const int y = rem / sp.nx, x = rem - y * sp.nx;
    int dir;
    const size_t idx = aa_slot(sp, sp.aa_layout, i, x, y, z, dir);
    a = ldpop<St>(f, (size_t)dir * sp.P + idx, i, 0, sp.ref_half, ph);
    b = ldpop<St>(f, (size_t)(Q + dir) * sp.P + idx, i, 1, sp.ref_half, ph);
}
// Current colour field of node n as the deviation references need it (0 otherwise).
template <class St>
__device__ inline float ref_phi(const float* phi_cur, size_t n) {
    return St::DEV ? phi_cur[n] : 0.0f;
}

// Fields of the current state. rho_k = sum_i f_i^k of the stored (post-collision)
// populations, which equals the post-stream density of the last step; the stored
// momentum is j + F, so u = (sum_i c_i f_i - F/2)/rho; F is re-evaluated from the
// two colour-field buffers exactly as the step did (have_force = 0 before a step).
template <class St>
__global__ void export_fields_kernel(const typename St::T* f, StepParams sp, int have_force,
                                     const float* phi_now, const float* sc_rho, double* rho_r,
                                     double* rho_b, double* u, double* phi) {
    // (node indices in 32 bits: a lattice has fewer than 2^31 nodes)
    const unsigned N = (unsigned)sp.N, plane = (unsigned)sp.nx * (unsigned)sp.ny;
    for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const unsigned zu = n / plane, rem = n - zu * plane;
        const unsigned yu = rem / (unsigned)sp.nx;
        const int x = (int)(rem - yu * (unsigned)sp.nx), y = (int)yu, z = (int)zu;
        const size_t q = pidx(sp.pitch, sp.nyp, sp.padx, x, y, z);
        const float ph = ref_phi<St>(phi_now, n);
        float rr = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            ldnode<St>(f, sp, n, q, i, ph, a, b);
            rr += a;
            rb += b;
            jx += cx(i) * (a + b);
            jy += cy(i) * (a + b);
            jz += cz(i) * (a + b);
        }
        float Fx = 0.f, Fy = 0.f, Fz = 0.f;
        if (have_force) {
            Fx = sp.fx_row[y];
            Fy = sp.gy;
            Fz = sp.gz;
            if (sp.A_nc > 0.0f) {
                // A_h of the last step (re-measured on its lag field before this kernel)
                // times the gradient of the last step's colour field
                float Gx, Gy, Gz;
                gradient_global(sp, phi_now, x, y, z, Gx, Gy, Gz);
                const float ah = sp.ah[n];
                Fx += ah * Gx;
                Fy += ah * Gy;
                Fz += ah * Gz;
            }
            if (sc_rho) {
                // Shan-Chen cohesive forces of the last step, from its densities
                // ([2][N]: red, blue): F^r + F^b = -(G/3)(rho_r S_b + rho_b S_r), S_k the
                // stencil 3 sum_i w_i rho_k(x + c_i) c_i
                float Sr[3], Sb[3];
                gradient_global(sp, sc_rho, x, y, z, Sr[0], Sr[1], Sr[2]);
                gradient_global(sp, sc_rho + N, x, y, z, Sb[0], Sb[1], Sb[2]);
                const float g3 = -sp.G_sc * (1.0f / 3.0f);
                Fx += rr * (g3 * Sb[0]) + rb * (g3 * Sr[0]);
                Fy += rr * (g3 * Sb[1]) + rb * (g3 * Sr[1]);
                Fz += rr * (g3 * Sb[2]) + rb * (g3 * Sr[2]);
            }
        }
        if (rho_r) rho_r[n] = rr;
        if (rho_b) rho_b[n] = rb;
        if (u) {
            const double inv_rho = 1.0 / ((double)rr + (double)rb);
            u[n] = ((double)jx - 0.5 * Fx) * inv_rho;
            u[N + n] = ((double)jy - 0.5 * Fy) * inv_rho;
            u[2 * (size_t)N + n] = ((double)jz - 0.5 * Fz) * inv_rho;
        }
        if (phi) phi[n] = phi_now[n];
    }
}

// Species densities of the stored state ([2][N] floats), summed as the export does.
template <class St>
__global__ void densities_kernel(const typename St::T* f, StepParams sp, const float* phi_now,
                                 float* rho) {
    const size_t N = sp.N, P = sp.P;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const size_t q = node_pidx(sp, n);
        const float ph = ref_phi<St>(phi_now, n);
        float rr = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            ldnode<St>(f, sp, n, q, i, ph, a, b);
            rr += a;
            rb += b;
        }
        rho[n] = rr;
        rho[N + n] = rb;
    }
}

template <class St>
__global__ void pops_to_f64_kernel(const typename St::T* f, StepParams sp, const float* phi_cur,
                                   double* fr, double* fb) {
    const size_t N = sp.N, P = sp.P;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const size_t q = node_pidx(sp, n);
        const float ph = ref_phi<St>(phi_cur, n);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            ldnode<St>(f, sp, n, q, i, ph, a, b);
            fr[(size_t)i * N + n] = a;
            fb[(size_t)i * N + n] = b;
        }
    }
}

// Populations and current colour field of the sub-box (x0, y0, z0) + [0, wx) x
// [0, wy) x [0, wz), wrapped on periodic axes, into out = {f_r [19][M], f_b [19][M],
// phi [M]}, M = wx wy wz (box index x fastest).
template <class St>
__global__ void window_kernel(const typename St::T* f, StepParams sp, const float* phi_cur, int x0,
                              int y0, int z0, int wx, int wy, int wz, double* out) {
    const size_t M = (size_t)wx * wy * wz, P = sp.P;
    for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < M;
         m += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(m % wx), j = (int)((m / wx) % wy), k = (int)(m / ((size_t)wx * wy));
        const int x = wrap_near(x0 + i, sp.nx), y = wrap_near(y0 + j, sp.ny), z = wrap_near(z0 + k, sp.nz);
        const size_t n = ((size_t)z * sp.ny + y) * sp.nx + x;
        const size_t q = pidx(sp.pitch, sp.nyp, sp.padx, x, y, z);
        const float ph = ref_phi<St>(phi_cur, n);
#pragma unroll
        for (int d = 0; d < Q; ++d) {
            float a, b;
            ldnode<St>(f, sp, n, q, d, ph, a, b);
            out[(size_t)d * M + m] = a;
            out[(size_t)(Q + d) * M + m] = b;
        }
        out[(size_t)2 * Q * M + m] = phi_cur[n];
    }
}

template <class St>
__global__ void f64_to_pops_kernel(typename St::T* f, StepParams sp, const float* phi_cur,
                                   const double* fr, const double* fb) {
    const size_t N = sp.N, P = sp.P;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const size_t q = node_pidx(sp, n);
        const float ph = ref_phi<St>(phi_cur, n);
        if constexpr (St::RED) {
            // reduced form: totals, kappa_k = rho_k / rho, and m from the first moment
            // of the red excess d_i = f^r_i - kappa_r f_i: with d_i = w_i (c_i . m)/|c_i|,
            // sum_i d_i c_i = m sum_i (w_i/|c_i|) c_i c_i = m (1 + sqrt 2)/9. Exact for
            // every recoloured split (all states the step produces); other splits are
            // projected onto that form.
            double rr = 0, rb = 0;
            for (int i = 0; i < Q; ++i) {
                rr += fr[(size_t)i * N + n];
                rb += fb[(size_t)i * N + n];
            }
            const double kr = rr / (rr + rb), kb = rb / (rr + rb);
            double mx = 0, my = 0, mz = 0;
            for (int i = 0; i < Q; ++i) {
                const double a = fr[(size_t)i * N + n], t = a + fb[(size_t)i * N + n];
                const double d = a - kr * t;
                mx += cx(i) * d;
                my += cy(i) * d;
                mz += cz(i) * d;
                St::store(f, (size_t)i * P + q, (float)t, St::tot_ref(i, 2.0f * sp.ref_half));
            }
            const double inv = 9.0 / (1.0 + sqrt(2.0));
            St::store_coef(f, P, q, 0, (float)kr);
            St::store_coef(f, P, q, 1, (float)kb);
            St::store_coef(f, P, q, 2, (float)(mx * inv));
            St::store_coef(f, P, q, 3, (float)(my * inv));
            St::store_coef(f, P, q, 4, (float)(mz * inv));
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float hw = wgt(i) * sp.ref_half;
                const int d = wdir(sp, i);
                St::store(f, (size_t)d * P + q, (float)fr[(size_t)i * N + n], dev_ref(hw, ph, 0));
                St::store(f, (size_t)(Q + d) * P + q, (float)fb[(size_t)i * N + n], dev_ref(hw, ph, 1));
            }
        }
    }
}

__global__ void f64_to_f32_kernel(float* dst, const double* src, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (float)src[k];
}
__global__ void f32_to_f64_kernel(double* dst, const float* src, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (double)src[k];
}

// Block-level FP64 sum of NV values per thread into out[blockIdx.x * NV + v]:
// warp shuffles, then the warps of the block in index order (deterministic).
template <int NV>
__device__ inline void block_sum(double (&v)[NV], double* out) {
    __shared__ double sh[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
        out[blockIdx.x * NV + threadIdx.x] = s;
    }
}

// Second pass: one block sums the per-block partials in index order.
template <int NV>
__global__ void finish_sum_kernel(const double* part, int nblocks, double* out) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += part[b * NV + k];
    block_sum<NV>(v, out);
}

// Conserved totals (FP64): sum f^r, sum f^b, P.
template <class St>
__global__ void totals_kernel(const typename St::T* f, StepParams sp, const float* phi_cur,
                              double* part) {
    double v[5] = {0, 0, 0, 0, 0};
    const size_t N = sp.N, P = sp.P;
    const float ref_half = sp.ref_half;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const size_t q = node_pidx(sp, n);
        const float ph = ref_phi<St>(phi_cur, n);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float af, bf;
            ldnode<St>(f, sp, n, q, i, ph, af, bf);
            const double a = af, b = bf;
            v[0] += a;
            v[1] += b;
            v[2] += cx(i) * (a + b);
            v[3] += cy(i) * (a + b);
            v[4] += cz(i) * (a + b);
        }
    }
    block_sum<5>(v, part);
}

// Laplace measurement, pass 1: V = sum (1 + phi)/2 with phi from the populations.
template <class St>
__global__ void volume_kernel(const typename St::T* f, StepParams sp, const float* phi_cur,
                              double* part) {
    double v[1] = {0};
    const size_t N = sp.N, P = sp.P;
    const float ref_half = sp.ref_half;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const size_t q = node_pidx(sp, n);
        const float ph = ref_phi<St>(phi_cur, n);
        double rr = 0, rb = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            ldnode<St>(f, sp, n, q, i, ph, a, b);
            rr += a;
            rb += b;
        }
        v[0] += 0.5 * (1.0 + (rr - rb) / (rr + rb));
    }
    block_sum<1>(v, part);
}

// Pass 2: pressure sums and node counts inside r < R-3 and outside r > R+5.
template <class St>
__global__ void pressure_kernel(const typename St::T* f, lbm_params p, StepParams sp,
                                const float* phi_cur, double c0, double c1, double c2, double R,
                                double* part) {
    double v[4] = {0, 0, 0, 0};
    const size_t N = sp.N, P = sp.P;
    const float ref_half = sp.ref_half;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((size_t)p.nx * p.ny));
        double d[3] = {x - c0, y - c1, z - c2};
        const int nn[3] = {p.nx, p.ny, p.nz};
        const int per[3] = {1, !p.wall_y, !p.wall_z};
        for (int a = 0; a < 3; ++a)
            if (per[a]) {
                if (d[a] > 0.5 * nn[a]) d[a] -= nn[a];
                if (d[a] < -0.5 * nn[a]) d[a] += nn[a];
            }
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r < R - 3.0 || r > R + 5.0) {
            const size_t q = node_pidx(sp, n);
            const float ph = ref_phi<St>(phi_cur, n);
            double rho = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float a, b;
                ldnode<St>(f, sp, n, q, i, ph, a, b);
                rho += (double)a + (double)b;
            }
            if (r < R - 3.0) {
                v[0] += rho / 3.0;
                v[1] += 1;
            } else {
                v[2] += rho / 3.0;
                v[3] += 1;
            }
        }
    }
    block_sum<4>(v, part);
}

// Pin distance field, three separable min-plus passes over the cube of
// half-width r: d2 = min over pins in the cube of dx^2 + dy^2 + dz^2 (255 = none).
// Pass along one axis; src codes 255 as "no pin in range".
__global__ void pin_pass_kernel(const uint8_t* src, uint8_t* dst, lbm_params p, int axis, int r,
                                int first) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        int c[3] = {(int)(n % p.nx), (int)((n / p.nx) % p.ny), (int)(n / ((size_t)p.nx * p.ny))};
        const int nn[3] = {p.nx, p.ny, p.nz};
        const int walled = axis == 1 ? p.wall_y : (axis == 2 ? p.wall_z : 0);
        int best = 255;
        for (int d = -r; d <= r; ++d) {
            int q[3] = {c[0], c[1], c[2]};
            q[axis] += d;
            if (walled && (q[axis] < 0 || q[axis] >= nn[axis])) continue;
            q[axis] = wrapi(q[axis], nn[axis]);
            const uint8_t s = src[((size_t)q[2] * p.ny + q[1]) * p.nx + q[0]];
            int val;
            if (first) val = s ? 0 : 255;
            else val = s;
            if (val == 255) continue;
            val += d * d;
            if (val < best) best = val;
        }
        dst[n] = (uint8_t)best;
    }
}

int grid_for(size_t n, int num_sms) {
    size_t b = (n + kThreads - 1) / kThreads;
    size_t cap = (size_t)num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------- helpers
static size_t elem_bytes(int storage) { return (storage == 0 || storage == 3) ? 4 : 2; }
static bool reduced_form(int storage) { return storage == 3 || storage == 4; }
// Population blocks per copy: stored (2Q, or the reduced form's Q totals and five
// coefficient blocks) and streamed (loaded by the step kernel's tensor copies, with
// ghost copies on periodic axes).
static int stored_blocks(int storage) {
    return storage == 3 ? Q + StoreQ5::AUX_BLOCKS : (storage == 4 ? Q + StoreQ5H::AUX_BLOCKS : 2 * Q);
}
static int streamed_blocks(int storage) { return reduced_form(storage) ? Q : 2 * Q; }

// Padded population layout: two ghost columns left and right of each row, the row
// length a multiple of 16 bytes (TMA alignment); two ghost rows above and below.
struct PadLayout {
    int pitch, nyp, padx;
    size_t P;
};
static PadLayout pad_layout(const lbm_params& p) {
    const int per32 = (int)(32 / elem_bytes(p.storage));
    PadLayout L;
    L.padx = step_pad_x(p.storage);                     // 32 bytes of ghosts + padding
    L.pitch = (p.nx + 2 * L.padx + per32 - 1) / per32 * per32;   // 32-byte rows
    L.pitch = std::max(L.pitch, 80);                    // at least one staged box wide
    L.nyp = std::max(p.ny + 4, 18);                     // at least one staged box high
    L.P = (size_t)L.pitch * L.nyp * p.nz;
    return L;
}

static lbm_status validate(const lbm_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return LBM_EINVAL; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "nx, ny, nz must be >= 1"; return LBM_EINVAL; }
    if ((double)p->nx * p->ny * p->nz > 2147483647.0) { why = "lattice larger than 2^31-1 nodes"; return LBM_EINVAL; }
    if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5)) { why = "tau_r and tau_b must be > 1/2"; return LBM_EINVAL; }
    if (!(p->beta >= 0.0 && p->beta <= 1.0)) { why = "beta must be in [0, 1]"; return LBM_EINVAL; }
    if (!(p->sigma >= 0.0)) { why = "sigma must be >= 0"; return LBM_EINVAL; }
    if (!(p->A_nc >= 0.0) || !(p->h_min >= 0.0)) { why = "A_nc and h_min must be >= 0"; return LBM_EINVAL; }
    if (p->A_nc > 0.0 && !(p->h_min > 0.0)) { why = "h_min must be > 0 when A_nc > 0"; return LBM_EINVAL; }
    double hcut = p->h_cut > 0 ? p->h_cut : 2.0 * p->h_min;
    if (p->A_nc > 0.0 && !(hcut > p->h_min)) { why = "h_cut must exceed h_min"; return LBM_EINVAL; }
    if (p->A_nc > 0.0 && hcut > 9.0) { why = "h_cut must be <= 9 (film rays of at most 25 samples)"; return LBM_EINVAL; }
    if (p->storage < 0 || p->storage > 4) { why = "unknown storage"; return LBM_EINVAL; }
    if (!(std::fabs(p->wall_u) < 0.3)) { why = "|wall_u| must be < 0.3"; return LBM_EINVAL; }
    if (p->wall_u != 0.0 && !p->wall_y) { why = "wall_u needs walls at the y extremes (wall_y)"; return LBM_EINVAL; }
    if (p->model != 0 && p->model != 1) { why = "unknown model"; return LBM_EINVAL; }
    if (p->model == 1 && p->A_nc != 0.0) { why = "the near-contact force belongs to the colour-gradient model"; return LBM_EINVAL; }
    if (p->model == 1 && reduced_form(p->storage)) { why = "the reduced storage forms hold recoloured (colour-gradient) states only"; return LBM_EINVAL; }
    if (!std::isfinite(p->G_sc)) { why = "G_sc must be finite"; return LBM_EINVAL; }
    if ((p->storage == 1 || p->storage == 2 || p->storage == 4) && !(p->rho0 > 0.0)) { why = "rho0 must be > 0 for deviation storage"; return LBM_EINVAL; }
    if (p->wall_y && p->ny < 2 && p->A_nc > 0) { why = "walled axis needs >= 2 nodes with A_nc"; return LBM_EINVAL; }
    if (p->wall_z && p->nz < 2 && p->A_nc > 0) { why = "walled axis needs >= 2 nodes with A_nc"; return LBM_EINVAL; }
    if (p->inplace != 0 && p->inplace != 1) { why = "inplace must be 0 or 1"; return LBM_EINVAL; }
    if (p->inplace && (p->model != 0 || p->storage > 2 || p->wall_u != 0.0)) {
        why = "in-place storage: colour-gradient model, full storage forms, walls at rest";
        return LBM_EINVAL;
    }
    if (p->inplace && pad_layout(*p).P >= ((size_t)1 << 31)) {
        why = "in-place storage indexes a padded population block in 31 bits";
        return LBM_EINVAL;
    }
    return LBM_OK;
}

extern "C" size_t lbm_footprint_bytes(const lbm_params* p) {
    if (!p) return 0;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const PadLayout L = pad_layout(*p);
    const size_t copies = p->inplace ? 1 : 2;
    size_t b = copies * (size_t)stored_blocks(p->storage) * L.P * elem_bytes(p->storage) +
               2 * N * sizeof(float) + p->ny * sizeof(float);
    if (p->A_nc > 0.0) b += N * sizeof(float);   // the near-contact strength A_h
    return b;
}

extern "C" void lbm_velocity_set(int c[LBM_Q * 3]) {
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = cx(i);
        c[3 * i + 1] = cy(i);
        c[3 * i + 2] = cz(i);
    }
}

// Work split of the step kernel over the GPU's CTA slots (num_sms x CTAs per SM).
struct WorkSplit {
    int zparts, chain, band_k, band_h, grid;
};
static WorkSplit work_split(const lbm_params& p, int num_sms) {
    WorkSplit w{1, 0, 0, 0, 1};
    const int tx = step_tile_x(), ty = step_tile_y();
    const long long tiles = (long long)((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty);
    // z parts: one CTA (one per SM) marches one part of one tile. Pick the number of
    // parts that minimises waves x (planes per part + 2 halo planes + ~2 planes of
    // pipeline fill), the cost of a part-major launch.
    const int S = (num_sms > 0 ? num_sms : 1) * step_ctas_per_sm();
    int best_k = 1;
    double best = 1e300;
    for (int k = 1; k <= p.nz && k <= 4096; ++k) {
        const long long ctas = tiles * k;
        const long long waves = (ctas + S - 1) / S;
        const double cost = (double)waves * ((double)p.nz / k + 4.0);
        if (cost < best * 0.999) {
            best = cost;
            best_k = k;
        }
    }
    w.zparts = best_k;
    w.grid = (int)(tiles * best_k);
    // chain mode when one wave of whole parts would leave SMs unevenly loaded: every
    // CTA slot, with about w = nz tiles / slots planes each: k = slots / tiles bands
    // of h ~ w planes, one CTA per (band, tile), and the rest shared by the remaining
    // slots; of h near w the one whose busiest CTA has the fewest planes (counting
    // about one plane of pipeline fill per tile a CTA starts) is taken.
    const long long units = tiles * p.nz;
    if (tiles < S && units >= 8LL * S && tiles * best_k != S) {
        const int k = (int)(S / tiles);
        const double wsh = (double)units / (double)S;
        double best_cost = (double)p.nz / best_k + 1.0;   // part mode: one part per CTA
        for (int h = std::max(1, (int)std::floor(wsh) - 2); h <= (int)std::ceil(wsh) + 3; ++h) {
            const int r = p.nz - k * h;
            const long long R = S - (long long)k * tiles;
            if (r < 0 || (r > 0 && R <= 0)) continue;
            double cost = h + 1.0;
            if (r > 0) {
                const double rem = (double)r * tiles / (double)R;
                cost = std::max(cost, rem + std::ceil(rem / r) + 1.0);
            }
            if (cost < best_cost) {
                best_cost = cost;
                w.band_k = k;
                w.band_h = h;
                w.chain = (int)(r > 0 ? S : (long long)k * tiles);
            }
        }
        if (w.chain > 0) w.grid = w.chain;
    }
    return w;
}

extern "C" lbm_status lbm_work_split(const lbm_params* p, int num_sms, long long out[5]) {
    std::string why;
    if (!out || num_sms < 1) return fail(nullptr, LBM_EINVAL, "out is NULL or num_sms < 1");
    if (validate(p, why) != LBM_OK) return fail(nullptr, LBM_EINVAL, why);
    const WorkSplit w = work_split(*p, num_sms);
    out[0] = w.zparts;
    out[1] = w.chain;
    out[2] = w.band_k;
    out[3] = w.band_h;
    out[4] = w.grid;
    return LBM_OK;
}

static void fill_step_params(lbm_ctx* c) {
    const lbm_params& p = c->p;
    StepParams& s = c->sp;
    s.fx_row = c->fx_row;
    s.pin_d2 = c->pin_d2;
    s.gy = (float)p.g[1];
    s.gz = (float)p.g[2];
    s.wall_u6 = p.wall_y ? (float)(6.0 * p.wall_u) : 0.0f;
    s.model = p.model;
    s.G_sc = (float)p.G_sc;
    s.nx = p.nx;
    s.ny = p.ny;
    s.nz = p.nz;
    s.N = c->N;
    s.pitch = c->pitch;
    s.nyp = c->nyp;
    s.padx = c->padx;
    s.ghost_arrays = streamed_blocks(p.storage);
    s.plane_p = (size_t)c->pitch * c->nyp;
    s.P = c->P;
    s.wall_y = p.wall_y ? 1 : 0;
    s.wall_z = p.wall_z ? 1 : 0;
    s.var_tau = p.tau_r != p.tau_b;
    s.omega0 = (float)(1.0 / p.tau_r);
    s.inv_nu_r = (float)(3.0 / (p.tau_r - 0.5));
    s.inv_nu_b = (float)(3.0 / (p.tau_b - 0.5));
    s.sigma = (float)p.sigma;
    s.beta = (float)p.beta;
    const double hcut = p.h_cut > 0 ? p.h_cut : 2.0 * p.h_min;
    s.A_nc = (float)p.A_nc;
    s.h_min = (float)p.h_min;
    s.h_cut = (float)hcut;
    const double b3 = p.A_nc > 0 ? std::pow(p.h_min / hcut, 3.0) : 0.0;
    s.ah_b3 = (float)b3;
    s.ah_inv = (float)(1.0 / (1.0 - b3));
    s.nsamp = (int)std::floor(2.0 * (hcut + 3.0)) + 1;
    s.ref_half = (p.storage == 1 || p.storage == 2 || p.storage == 4) ? (float)(0.5 * p.rho0) : 0.0f;
    const int tx = step_tile_x(), ty = step_tile_y();
    s.tiles_x = (p.nx + tx - 1) / tx;
    s.tiles_y = (p.ny + ty - 1) / ty;
    s.err = c->err_word;
    s.aa_layout = c->aa ? c->layout : -1;
    s.nc_seg = nc_segment_blocks(p.nx, p.ny, p.nz, c->num_sms);
    s.ah = c->ah;
    const WorkSplit w = work_split(p, c->num_sms);
    s.zparts = w.zparts;
    s.chain = w.chain;
    s.band_k = w.band_k;
    s.band_h = w.band_h;
    c->grid = w.grid;
}

// The step kernel's bounded waits record a give-up in a device word; report it.
static lbm_status check_err_word(lbm_ctx* c) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->err_word, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, LBM_ETIMEOUT, "a bounded wait in the step kernel gave up");
    return LBM_OK;
}

namespace lbm {
void step_params_ahead(const lbm_ctx* c, int ahead, int zparts, BatchLattice* out) {
    const int cur = c->cur ^ (ahead & 1), pc = c->pc ^ (ahead & 1);
    StepParams s = c->sp;
    s.fin = c->f[cur];
    s.fout = c->f[1 - cur];
    s.phi_lag = c->phi[pc];
    s.phi_out = c->phi[1 - pc];
    if (zparts > 0) {
        s.zparts = zparts;
        s.chain = 0;
        s.band_k = s.band_h = 0;
    }
    out->in_map = c->tmap[cur];
    out->out_map = c->smap[1 - cur];
    out->p = s;
    out->fout = c->f[1 - cur];
}
void nc_params_ahead(const lbm_ctx* c, int ahead, NcBatchLattice* out) {
    const int cur = c->cur ^ (ahead & 1), pc = c->pc ^ (ahead & 1);
    StepParams s = c->sp;
    s.fin = c->f[cur];
    s.fout = c->f[1 - cur];
    s.phi_lag = c->phi[pc];
    s.phi_out = c->phi[1 - pc];
    s.ghost_f = ghost_cells(s) > 0 ? c->f[cur] : nullptr;
    out->lag_map = c->phimap[pc];
    out->tma_ok = c->phimap_ok ? 1 : 0;
    out->p = s;
}
double ctx_h_cut(const lbm_ctx* c) { return c->p.h_cut > 0 ? c->p.h_cut : 2.0 * c->p.h_min; }
void advance_state(lbm_ctx* c, long long k) {
    if (k & 1) {
        c->cur ^= 1;
        c->pc ^= 1;
    }
    c->steps += k;
}
lbm_status check_errors(lbm_ctx* c) { return check_err_word(c); }
int ctx_num_sms(const lbm_ctx* c) { return c->num_sms; }
cudaStream_t ctx_stream(const lbm_ctx* c) { return c->stream; }
}  // namespace lbm

// ---------------------------------------------------------------- API
extern "C" lbm_status lbm_create(const lbm_params* p, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (validate(p, why) != LBM_OK) return fail(nullptr, LBM_EINVAL, why);
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->p = *p;
    c->N = (size_t)p->nx * p->ny * p->nz;
    c->elem = elem_bytes(p->storage);
    c->stream = (cudaStream_t)p->cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBM_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    const PadLayout L = pad_layout(*p);
    c->pitch = L.pitch;
    c->nyp = L.nyp;
    c->padx = L.padx;
    c->P = L.P;
    const size_t pop_bytes = (size_t)stored_blocks(p->storage) * c->P * c->elem;
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        return cudaMalloc(ptr, bytes) == cudaSuccess;
    };
    c->aa = p->inplace != 0;
    bool ok = alloc(&c->f[0], pop_bytes) && (c->aa || alloc(&c->f[1], pop_bytes)) &&
              alloc((void**)&c->phi[0], c->N * sizeof(float)) &&
              alloc((void**)&c->phi[1], c->N * sizeof(float)) &&
              alloc((void**)&c->fx_row, p->ny * sizeof(float)) &&
              alloc((void**)&c->err_word, sizeof(int)) &&
              (p->A_nc > 0.0 ? alloc((void**)&c->ah, c->N * sizeof(float)) : true);
    c->red_blocks = c->num_sms * 8;
    ok = ok && alloc((void**)&c->red, (size_t)(c->red_blocks + 1) * 8 * sizeof(double));
    ok = ok && cudaMallocHost((void**)&c->red_host, 8 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbm_destroy(c);
        return fail(nullptr, LBM_ENOMEM, "device allocation failed");
    }
    // body force per row, evaluated in FP64 on the host
    float* row = new (std::nothrow) float[p->ny];
    if (!row) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    }
    for (int y = 0; y < p->ny; ++y)
        row[y] = (float)(p->g[0] + p->kolmogorov_amp * std::sin(2.0 * M_PI * (double)y / (double)p->ny));
    e = cudaMemcpy(c->fx_row, row, p->ny * sizeof(float), cudaMemcpyHostToDevice);
    delete[] row;
    if (e == cudaSuccess) e = cudaMemset(c->err_word, 0, sizeof(int));
    // colour fields start at 0, so deviation storage has a finite reference even when
    // populations are set before any field
    if (e == cudaSuccess) e = cudaMemset(c->phi[0], 0, c->N * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->phi[1], 0, c->N * sizeof(float));
    if (e != cudaSuccess) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    }
    // TMA descriptors of the two population copies: 4-D [blocks][nz][nyp][pitch], boxes
    // of BW x (TY+2) x 1 x 1 elements, zero fill outside; loads cover the streamed
    // blocks, stores every stored block
    {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) {
            lbm_destroy(c);
            return fail(nullptr, LBM_ECUDA, "cuTensorMapEncodeTiled unavailable");
        }
        auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        const cuuint64_t dims[4] = {(cuuint64_t)c->pitch, (cuuint64_t)c->nyp, (cuuint64_t)p->nz,
                                    (cuuint64_t)streamed_blocks(p->storage)};
        const cuuint64_t strides[3] = {(cuuint64_t)c->pitch * c->elem,
                                       (cuuint64_t)c->pitch * c->nyp * c->elem,
                                       (cuuint64_t)c->P * c->elem};
        const cuuint32_t box[4] = {(cuuint32_t)step_box_width(p->storage), (cuuint32_t)step_box_rows(), 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUtensorMapDataType dt = c->elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT16;
        // store maps end at the interior (x < nx, y < ny), so the tile stores of edge
        // tiles are clipped there and never touch ghost or padding cells
        const cuuint64_t sdims[4] = {(cuuint64_t)(c->padx + p->nx), (cuuint64_t)(2 + p->ny),
                                     (cuuint64_t)p->nz, (cuuint64_t)stored_blocks(p->storage)};
        const cuuint32_t sbox[4] = {(cuuint32_t)step_tile_x(), (cuuint32_t)step_tile_y(), 1, 1};
        for (int b = 0; b < (c->aa ? 0 : 2); ++b) {   // (in-place steps need no tensor maps)
            CUresult r = encode(&c->tmap[b], dt, 4, c->f[b], dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r == CUDA_SUCCESS)
                r = encode(&c->smap[b], dt, 4, c->f[b], sdims, strides, sbox, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                lbm_destroy(c);
                return fail(nullptr, LBM_ECUDA, "cuTensorMapEncodeTiled failed");
            }
        }
        // the near-contact pass copies the planes of its halo cubes from a colour field
        // (3-D, x fastest) with one tensor copy per plane where the cube lies inside the
        // lattice in x and y: rows must be a multiple of 16 bytes long, and the lattice
        // at least a cube wide in x and y
        if (p->A_nc > 0.0 && p->nx % 4 == 0) {
            int box[3];
            nc_cube_box(p->h_cut > 0 ? p->h_cut : 2.0 * p->h_min, box);
            if (p->nx >= box[0] && p->ny >= box[1]) {
                const cuuint64_t pd[3] = {(cuuint64_t)p->nx, (cuuint64_t)p->ny, (cuuint64_t)p->nz};
                const cuuint64_t ps[2] = {(cuuint64_t)p->nx * sizeof(float),
                                          (cuuint64_t)p->nx * p->ny * sizeof(float)};
                const cuuint32_t pb[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
                const cuuint32_t pe[3] = {1, 1, 1};
                bool ok = true;
                for (int b = 0; b < 2 && ok; ++b)
                    ok = encode(&c->phimap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->phi[b], pd, ps,
                                pb, pe, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
                c->phimap_ok = ok;
            }
        }
    }
    fill_step_params(c);
    *out = c;
    return LBM_OK;
}

extern "C" void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->phi[0]);
    cudaFree(c->phi[1]);
    cudaFree(c->fx_row);
    cudaFree(c->pin_d2);
    cudaFree(c->pin_mask);
    cudaFree(c->stage);
    cudaFree(c->red);
    cudaFree(c->err_word);
    cudaFree(c->ah);
    if (c->red_host) cudaFreeHost(c->red_host);
    delete c;
}

extern "C" const char* lbm_last_error(const lbm_ctx* c) {
    return c ? c->err.c_str() : g_create_err.c_str();
}

// FP64 staging of at least `doubles` values (grown on demand; the old contents are
// not kept). Calls that only exchange fields need 7N, population calls 2QN.
static lbm_status ensure_stage(lbm_ctx* c, size_t doubles) {
    if (c->stage && c->stage_cap >= doubles) return LBM_OK;
    if (c->stage) {
        cudaStreamSynchronize(c->stream);   // queued work may still read the old buffer
        cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_cap = 0;
    }
    if (cudaMalloc((void**)&c->stage, doubles * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LBM_ENOMEM, "staging allocation failed");
    }
    c->stage_cap = doubles;
    return LBM_OK;
}

namespace lbm {
lbm_status ctx_stage(lbm_ctx* c, size_t doubles) { return ensure_stage(c, doubles); }
lbm_status ctx_fail(lbm_ctx* c, lbm_status s, const std::string& msg) { return fail(c, s, msg); }
}  // namespace lbm

template <class F>
static void dispatch(int storage, F&& fn) {
    if (storage == 0) fn(StoreF32{});
    else if (storage == 1) fn(StoreF16{});
    else if (storage == 2) fn(StoreBF16{});
    else if (storage == 3) fn(StoreQ5{});
    else fn(StoreQ5H{});
}

// Device address of a host buffer that kernels may read and write directly (pinned host
// memory mapped into the device's address space, e.g. from cudaHostAlloc), else null.
static void* mapped_host(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
// The device addresses of the given (non-null) host buffers when every one of them is
// mapped; false otherwise (the buffers then go through the staging buffer).
static bool map_all(const void* const* host, void** dev, int n) {
    for (int k = 0; k < n; ++k) {
        dev[k] = nullptr;
        if (host[k] && !(dev[k] = mapped_host(host[k]))) return false;
    }
    return true;
}

extern "C" lbm_status lbm_set_fields(lbm_ctx* c, const double* rho_r, const double* rho_b,
                                     const double* u, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!rho_r || !rho_b) return fail(c, LBM_EINVAL, "rho_r and rho_b are required");
    const size_t N = c->N;
    const double *dr = rho_r, *db = rho_b, *du = u;
    // host buffers mapped into the device's address space are read by the kernel
    // directly; any other host buffer is copied to the staging buffer first
    bool staged = !on_device;
    if (!on_device) {
        const void* hp[3] = {rho_r, rho_b, u};
        void* dv[3];
        if (map_all(hp, dv, 3)) {
            dr = static_cast<const double*>(dv[0]);
            db = static_cast<const double*>(dv[1]);
            du = static_cast<const double*>(dv[2]);
            staged = false;
        }
    }
    if (staged) {
        // (sized for lbm_get_fields too, the usual next host exchange, so that the
        // buffer is not freed and allocated again there)
        if (ensure_stage(c, 7 * c->N) != LBM_OK) return LBM_ENOMEM;
        CK(c, cudaMemcpyAsync(c->stage, rho_r, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->stage + N, rho_b, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        dr = c->stage;
        db = c->stage + N;
        if (u) {
            CK(c, cudaMemcpyAsync(c->stage + 2 * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            du = c->stage + 2 * N;
        }
    }
    const int grid = grid_for(N, c->num_sms);
    c->cur = 0;
    c->pc = 0;
    if (c->aa) {                 // in-place storage starts in the slot layout 0
        c->layout = 0;
        c->sp.aa_layout = 0;
    }
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        init_fields_kernel<St><<<grid, kThreads, 0, c->stream>>>(
            (typename St::T*)c->f[0], c->phi[0], c->phi[1], dr, db, du, c->sp);
    });
    CK(c, cudaGetLastError());
    if (!c->aa) CK(c, launch_ghost_fill(c->f[0], c->sp, c->p.storage, c->num_sms, c->stream));
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));  // host arrays may be freed
    c->steps = 0;
    c->fields_set = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_pin_mask(lbm_ctx* c, const uint8_t* mask, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!mask) {
        cudaFree(c->pin_d2);
        c->pin_d2 = nullptr;
        fill_step_params(c);
        return LBM_OK;
    }
    const size_t N = c->N;
    if (!c->pin_d2) {
        if (cudaMalloc((void**)&c->pin_d2, N) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LBM_ENOMEM, "pin allocation failed");
        }
    }
    if (!c->pin_mask) {
        if (cudaMalloc((void**)&c->pin_mask, N) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LBM_ENOMEM, "pin allocation failed");
        }
    }
    CK(c, cudaMemcpyAsync(c->pin_mask, mask, N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    const double hcut = c->p.h_cut > 0 ? c->p.h_cut : 2.0 * c->p.h_min;
    const int r = (int)std::ceil(hcut);
    if (3 * r * r >= 255) return fail(c, LBM_EINVAL, "h_cut too large for pinning sites (<= 9)");
    const int grid = grid_for(N, c->num_sms);
    // x pass: mask -> d2 ; y pass: d2 -> mask buffer ; z pass: mask buffer -> d2
    pin_pass_kernel<<<grid, kThreads, 0, c->stream>>>(c->pin_mask, c->pin_d2, c->p, 0, r, 1);
    pin_pass_kernel<<<grid, kThreads, 0, c->stream>>>(c->pin_d2, c->pin_mask, c->p, 1, r, 0);
    pin_pass_kernel<<<grid, kThreads, 0, c->stream>>>(c->pin_mask, c->pin_d2, c->p, 2, r, 0);
    CK(c, cudaGetLastError());
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->pin_mask);
    c->pin_mask = nullptr;
    fill_step_params(c);
    return LBM_OK;
}

// Launches of one time step: the near-contact pass (A_nc > 0), which writes every
// node's A_h from the lagged colour field, the step kernel and, without near-contact
// force, the ghost-copy fill of the step's output (with it, the next pass writes those
// ghost copies). Events (optional) bracket the launches: e0 .. e1 pass, e1 .. e2 step
// kernel, e2 .. e3 ghost fill.
static cudaError_t launch_one_step(lbm_ctx* c, cudaEvent_t e0, cudaEvent_t e1, cudaEvent_t e2,
                                   cudaEvent_t e3 = nullptr) {
    StepParams s = c->sp;
    s.fin = c->f[c->cur];
    s.fout = c->f[1 - c->cur];
    s.phi_lag = c->phi[c->pc];
    s.phi_out = c->phi[1 - c->pc];
    const bool nc = c->p.A_nc > 0.0;
    cudaError_t e = cudaSuccess;
    if (c->aa) {
        // in place: the pass, then the colour-field and collide passes over the one copy
        s.fin = s.fout = c->f[0];
        s.ghost_f = nullptr;
        if (e0) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess && nc)
            e = launch_nc_block(s, c->phimap[c->pc], c->phimap_ok, c->p.storage, c->num_sms,
                                c->stream);
        if (e == cudaSuccess && e1) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = launch_aa_step(s, c->layout, c->p.storage, c->num_sms, c->stream);
        if (e == cudaSuccess && e2) e = cudaEventRecord(e2, c->stream);
        if (e == cudaSuccess && e3) e = cudaEventRecord(e3, c->stream);
        if (e != cudaSuccess) return e;
        c->layout ^= 1;
        c->sp.aa_layout = c->layout;
        c->pc ^= 1;
        c->steps++;
        return cudaSuccess;
    }
    if (e0) e = cudaEventRecord(e0, c->stream);
    if (nc) {
        s.ghost_f = ghost_cells(s) > 0 ? c->f[c->cur] : nullptr;
        if (e == cudaSuccess)
            e = launch_nc_block(s, c->phimap[c->pc], c->phimap_ok, c->p.storage, c->num_sms,
                                c->stream);
    }
    if (e == cudaSuccess && e1) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess)
        e = launch_step(s, c->tmap[c->cur], c->smap[1 - c->cur], c->p.storage, c->grid, c->stream);
    if (e == cudaSuccess && e2) e = cudaEventRecord(e2, c->stream);
    // ghost copies of the periodic axes for the next step's halo loads
    if (e == cudaSuccess && !nc)
        e = launch_ghost_fill(c->f[1 - c->cur], s, c->p.storage, c->num_sms, c->stream);
    if (e == cudaSuccess && e3) e = cudaEventRecord(e3, c->stream);
    if (e != cudaSuccess) return e;
    c->cur ^= 1;
    c->pc ^= 1;
    c->steps++;
    return cudaSuccess;
}

extern "C" lbm_status lbm_step(lbm_ctx* c, int n) {
    if (!c) return LBM_EINVAL;
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    nvtxRangePushA("lbm_step");   // host-side range over the launches of the n steps
    for (int t = 0; t < n; ++t) {
        cudaError_t e = launch_one_step(c, nullptr, nullptr, nullptr);
        if (e != cudaSuccess) {
            nvtxRangePop();
            return cuda_fail(c, e, "step launch");
        }
    }
    nvtxRangePop();
    return LBM_OK;
}

extern "C" lbm_status lbm_step_timed(lbm_ctx* c, int n, double out_ms[3]) {
    if (!c || !out_ms) return LBM_EINVAL;
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    out_ms[0] = out_ms[1] = out_ms[2] = 0.0;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) CK(c, cudaEventCreate(&ev[k]));
    lbm_status st = LBM_OK;
    for (int t = 0; t < n && st == LBM_OK; ++t) {
        cudaError_t e = launch_one_step(c, ev[0], ev[1], ev[2], ev[3]);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        float a = 0.f, b = 0.f, g = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&g, ev[2], ev[3]);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "timed step");
            break;
        }
        out_ms[0] += a;
        out_ms[1] += b;
        out_ms[2] += g;
    }
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    if (st != LBM_OK) return st;
    return check_err_word(c);
}

// A near-contact pass outside the time step (diagnostics): A_h of s.phi_lag into s.ah,
// touching none of the live step state.
static cudaError_t diag_pass(lbm_ctx* c, StepParams s) {
    s.ghost_f = nullptr;
    const int k = s.phi_lag == c->phi[0] ? 0 : 1;
    const bool tma = c->phimap_ok && s.phi_lag == c->phi[k];
    return launch_nc_block(s, c->phimap[k], tma, c->p.storage, c->num_sms, c->stream);
}

extern "C" lbm_status lbm_get_fields(lbm_ctx* c, double* rho_r, double* rho_b, double* u,
                                     double* phi, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    const size_t N = c->N;
    double *dr = rho_r, *db = rho_b, *du = u, *dp = phi;
    // host buffers mapped into the device's address space are written by the export
    // kernel directly (no staging copy); any other host buffer goes through staging
    bool staged = !on_device;
    if (!on_device) {
        const void* hp[4] = {rho_r, rho_b, u, phi};
        void* dv[4];
        if (map_all(hp, dv, 4)) {
            dr = static_cast<double*>(dv[0]);
            db = static_cast<double*>(dv[1]);
            du = static_cast<double*>(dv[2]);
            dp = static_cast<double*>(dv[3]);
            staged = false;
        }
    }
    if (staged) {
        if (ensure_stage(c, 7 * N) != LBM_OK) return LBM_ENOMEM;
        dr = rho_r ? c->stage : nullptr;
        db = rho_b ? c->stage + N : nullptr;
        du = u ? c->stage + 2 * N : nullptr;
        dp = phi ? c->stage + 5 * N : nullptr;
    }
    StepParams s = c->sp;
    s.phi_lag = c->phi[1 - c->pc];   // the lag field the last step's rays read
    const int grid = grid_for(N, c->num_sms);
    if (c->steps > 0 && c->p.A_nc > 0.0) {
        // A_h of the last step, re-measured on its lag field, into the A_h buffer: every
        // step's near-contact pass writes all of it before the step reads it, so between
        // steps it holds nothing the state depends on
        s.ah = c->ah;
        CK(c, diag_pass(c, s));
    }
    float* sc_rho = nullptr;
    if (c->steps > 0 && c->p.model == 1 && u) {
        // densities of the last step for its cohesive forces (2N floats), in scratch
        // space after the staged fields, or at the start of the staging buffer
        if (ensure_stage(c, staged ? 7 * N : N) != LBM_OK) return LBM_ENOMEM;
        sc_rho = reinterpret_cast<float*>(c->stage + (staged ? 6 * N : 0));
        dispatch(c->p.storage, [&](auto st) {
            using St = decltype(st);
            densities_kernel<St><<<grid, kThreads, 0, c->stream>>>(
                (const typename St::T*)c->f[c->cur], s, c->phi[c->pc], sc_rho);
        });
    }
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        export_fields_kernel<St><<<grid, kThreads, 0, c->stream>>>(
            (const typename St::T*)c->f[c->cur], s, c->steps > 0 ? 1 : 0, c->phi[c->pc], sc_rho,
            dr, db, du, dp);
    });
    CK(c, cudaGetLastError());
    if (staged) {
        if (rho_r) CK(c, cudaMemcpyAsync(rho_r, dr, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (rho_b) CK(c, cudaMemcpyAsync(rho_b, db, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (u) CK(c, cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (phi) CK(c, cudaMemcpyAsync(phi, dp, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_nc_field(lbm_ctx* c, double* ah, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    if (!ah) return fail(c, LBM_EINVAL, "ah is required");
    const size_t N = c->N;
    if (ensure_stage(c, 7 * N) != LBM_OK) return LBM_ENOMEM;
    const int grid = grid_for(N, c->num_sms);
    float* scratch = reinterpret_cast<float*>(c->stage + 6 * N);
    if (c->p.A_nc > 0.0) {
        // measured in scan mode on the current colour field (the next step's lag
        // field) into scratch; the live A_h buffer is untouched
        StepParams s = c->sp;
        s.phi_lag = c->phi[c->pc];
        s.ah = scratch;
        CK(c, diag_pass(c, s));
    } else {
        CK(c, cudaMemsetAsync(scratch, 0, N * sizeof(float), c->stream));
    }
    double* dst = on_device ? ah : c->stage;
    f32_to_f64_kernel<<<grid, kThreads, 0, c->stream>>>(dst, scratch, N);
    CK(c, cudaGetLastError());
    if (!on_device) CK(c, cudaMemcpyAsync(ah, dst, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_selftest_timeout(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    CK(c, cudaMemsetAsync(c->err_word, 0, sizeof(int), c->stream));
    CK(c, launch_wait_selftest(c->err_word, c->stream));
    const lbm_status st = check_err_word(c);
    CK(c, cudaMemsetAsync(c->err_word, 0, sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (st == LBM_ETIMEOUT) {
        c->err.clear();
        return LBM_ETIMEOUT;
    }
    return st == LBM_OK ? fail(c, LBM_OK, "the bounded wait did not give up") : st;
}

extern "C" lbm_status lbm_get_pops(lbm_ctx* c, double* f_r, double* f_b, double* phi_lag,
                                   int on_device) {
    if (!c) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    if (!f_r || !f_b) return fail(c, LBM_EINVAL, "f_r and f_b are required");
    const size_t N = c->N;
    double *dr = f_r, *db = f_b;
    if (!on_device) {
        if (ensure_stage(c, 2 * Q * N) != LBM_OK) return LBM_ENOMEM;
        dr = c->stage;
        db = c->stage + Q * N;
    }
    const int grid = grid_for(N, c->num_sms);
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        pops_to_f64_kernel<St><<<grid, kThreads, 0, c->stream>>>(
            (const typename St::T*)c->f[c->cur], c->sp, c->phi[c->pc], dr, db);
    });
    CK(c, cudaGetLastError());
    if (!on_device) {
        CK(c, cudaMemcpyAsync(f_r, dr, Q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemcpyAsync(f_b, db, Q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    if (phi_lag) {
        // the lag buffer of the next step is the colour field of the last step
        if (on_device) {
            f32_to_f64_kernel<<<grid, kThreads, 0, c->stream>>>(phi_lag, c->phi[c->pc], N);
            CK(c, cudaGetLastError());
        } else {
            CK(c, cudaStreamSynchronize(c->stream));
            f32_to_f64_kernel<<<grid, kThreads, 0, c->stream>>>(c->stage, c->phi[c->pc], N);
            CK(c, cudaGetLastError());
            CK(c, cudaMemcpyAsync(phi_lag, c->stage, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        }
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_window(lbm_ctx* c, int x0, int y0, int z0, int wx, int wy, int wz,
                                     double* f_r, double* f_b, double* phi_lag, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    if (!f_r || !f_b) return fail(c, LBM_EINVAL, "f_r and f_b are required");
    const lbm_params& p = c->p;
    if (wx < 1 || wy < 1 || wz < 1 || wx > p.nx || wy > p.ny || wz > p.nz)
        return fail(c, LBM_EINVAL, "window extents must be in [1, n] per axis");
    if ((p.wall_y && (y0 < 0 || y0 + wy > p.ny)) || (p.wall_z && (z0 < 0 || z0 + wz > p.nz)))
        return fail(c, LBM_EINVAL, "window must lie inside the lattice along walled axes");
    const size_t M = (size_t)wx * wy * wz, total = (2 * Q + 1) * M;
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, total * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LBM_ENOMEM, "window staging allocation failed");
    }
    const int grid = grid_for(M, c->num_sms);
    dispatch(p.storage, [&](auto st) {
        using St = decltype(st);
        window_kernel<St><<<grid, kThreads, 0, c->stream>>>((const typename St::T*)c->f[c->cur], c->sp,
                                                            c->phi[c->pc], x0, y0, z0, wx, wy, wz, buf);
    });
    cudaError_t e = cudaGetLastError();
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_r, buf, Q * M * sizeof(double), kind, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_b, buf + Q * M, Q * M * sizeof(double), kind, c->stream);
    if (e == cudaSuccess && phi_lag)
        e = cudaMemcpyAsync(phi_lag, buf + 2 * Q * M, M * sizeof(double), kind, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_window");
    return LBM_OK;
}

// Z-plane ranges of the stored state (slab decomposition): every stored block's
// planes, then the lagged colour field's, copied as stored.
extern "C" size_t lbm_planes_bytes(const lbm_ctx* c, int h) {
    if (!c || h < 1) return 0;
    const size_t plane_p = (size_t)c->pitch * c->nyp;
    return (size_t)stored_blocks(c->p.storage) * h * plane_p * c->elem +
           (size_t)h * c->p.nx * c->p.ny * sizeof(float);
}

static lbm_status planes_copy(lbm_ctx* c, int z0, int h, void* buf, bool get) {
    if (!c) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    if (!buf) return fail(c, LBM_EINVAL, "buf is NULL");
    if (h < 1 || z0 < 0 || z0 + h > c->p.nz) return fail(c, LBM_EINVAL, "planes outside the lattice");
    if (c->aa) return fail(c, LBM_EINVAL, "in-place storage keeps a node's populations in its neighbours' planes");
    const size_t plane_p = (size_t)c->pitch * c->nyp;
    const size_t seg = (size_t)h * plane_p * c->elem;   // bytes per block
    unsigned char* b = static_cast<unsigned char*>(buf);
    unsigned char* f = static_cast<unsigned char*>(c->f[c->cur]);
    const int blocks = stored_blocks(c->p.storage);
    for (int k = 0; k < blocks; ++k) {
        unsigned char* blk = f + ((size_t)k * c->P + (size_t)z0 * plane_p) * c->elem;
        CK(c, cudaMemcpyAsync(get ? b + k * seg : blk, get ? blk : b + k * seg, seg,
                              cudaMemcpyDeviceToDevice, c->stream));
    }
    const size_t plane = (size_t)c->p.nx * c->p.ny;
    float* ph = c->phi[c->pc] + (size_t)z0 * plane;
    unsigned char* pb = b + blocks * seg;
    CK(c, cudaMemcpyAsync(get ? (void*)pb : (void*)ph, get ? (const void*)ph : (const void*)pb,
                          (size_t)h * plane * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return LBM_OK;
}
extern "C" lbm_status lbm_get_planes(lbm_ctx* c, int z0, int h, void* buf) {
    return planes_copy(c, z0, h, buf, true);
}
extern "C" lbm_status lbm_set_planes(lbm_ctx* c, int z0, int h, const void* buf) {
    return planes_copy(c, z0, h, const_cast<void*>(buf), false);
}

extern "C" lbm_status lbm_set_pops(lbm_ctx* c, const double* f_r, const double* f_b,
                                   const double* phi_lag, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!f_r || !f_b) return fail(c, LBM_EINVAL, "f_r and f_b are required");
    const size_t N = c->N;
    const int grid = grid_for(N, c->num_sms);
    if (!on_device && ensure_stage(c, 2 * Q * N) != LBM_OK) return LBM_ENOMEM;
    if (c->aa) {                 // in-place storage: the state is written in layout 0
        c->layout = 0;
        c->sp.aa_layout = 0;
    }
    // the colour field first: deviation storage encodes the populations against it
    if (phi_lag) {
        const double* src = phi_lag;
        if (!on_device) {
            CK(c, cudaMemcpyAsync(c->stage, phi_lag, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            src = c->stage;
        }
        f64_to_f32_kernel<<<grid, kThreads, 0, c->stream>>>(c->phi[c->pc], src, N);
        CK(c, cudaGetLastError());
    }
    const double *dr = f_r, *db = f_b;
    if (!on_device) {
        CK(c, cudaMemcpyAsync(c->stage, f_r, Q * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->stage + Q * N, f_b, Q * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        dr = c->stage;
        db = c->stage + Q * N;
    }
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        f64_to_pops_kernel<St><<<grid, kThreads, 0, c->stream>>>(
            (typename St::T*)c->f[c->cur], c->sp, c->phi[c->pc], dr, db);
    });
    CK(c, cudaGetLastError());
    if (!c->aa) CK(c, launch_ghost_fill(c->f[c->cur], c->sp, c->p.storage, c->num_sms, c->stream));
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    c->fields_set = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_observables(lbm_ctx* c, double out[8]) {
    if (!c || !out) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    const int grid = c->red_blocks;
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        totals_kernel<St><<<grid, kThreads, 0, c->stream>>>((const typename St::T*)c->f[c->cur],
                                                            c->sp, c->phi[c->pc], c->red);
    });
    finish_sum_kernel<5><<<1, kThreads, 0, c->stream>>>(c->red, grid, c->red + (size_t)grid * 8);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(c->red_host, c->red + (size_t)grid * 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 5; ++k) out[k] = c->red_host[k];
    out[5] = (double)c->steps;
    out[6] = out[7] = 0.0;
    return LBM_OK;
}

extern "C" lbm_status lbm_laplace(lbm_ctx* c, const double centre[3], double out[5]) {
    if (!c || !centre || !out) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    const int grid = c->red_blocks;
    double* fin = c->red + (size_t)grid * 8;
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        volume_kernel<St><<<grid, kThreads, 0, c->stream>>>((const typename St::T*)c->f[c->cur],
                                                             c->sp, c->phi[c->pc], c->red);
    });
    finish_sum_kernel<1><<<1, kThreads, 0, c->stream>>>(c->red, grid, fin);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(c->red_host, fin, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double V = c->red_host[0];
    const double R = std::cbrt(3.0 * V / (4.0 * M_PI));
    dispatch(c->p.storage, [&](auto st) {
        using St = decltype(st);
        pressure_kernel<St><<<grid, kThreads, 0, c->stream>>>(
            (const typename St::T*)c->f[c->cur], c->p, c->sp, c->phi[c->pc], centre[0], centre[1],
            centre[2], R, c->red);
    });
    finish_sum_kernel<4><<<1, kThreads, 0, c->stream>>>(c->red, grid, fin);
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(c->red_host, fin, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double* h = c->red_host;
    const double pin = h[1] > 0 ? h[0] / h[1] : NAN, pout = h[3] > 0 ? h[2] / h[3] : NAN;
    out[0] = pin - pout;
    out[1] = R;
    out[2] = pin;
    out[3] = pout;
    out[4] = V;
    return LBM_OK;
}

extern "C" size_t lbm_state_bytes(const lbm_ctx* c) {
    if (!c) return 0;
    return (size_t)stored_blocks(c->p.storage) * c->P * c->elem + 2 * c->N * sizeof(float) +
           2 * sizeof(long long);
}

extern "C" lbm_status lbm_save_state(lbm_ctx* c, void* host_buf) {
    if (!c || !host_buf) return LBM_EINVAL;
    if (!c->fields_set) return fail(c, LBM_ESTATE, "lbm_set_fields has not been called");
    char* b = (char*)host_buf;
    const size_t pb = (size_t)stored_blocks(c->p.storage) * c->P * c->elem, fb = c->N * sizeof(float);
    CK(c, cudaMemcpyAsync(b, c->f[c->cur], pb, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(b + pb, c->phi[c->pc], fb, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(b + pb + fb, c->phi[1 - c->pc], fb, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memcpy(b + pb + 2 * fb, &c->steps, sizeof(long long));
    const long long layout = c->aa ? c->layout : -1;   // in-place storage: the state's layout
    std::memcpy(b + pb + 2 * fb + sizeof(long long), &layout, sizeof(long long));
    return LBM_OK;
}

extern "C" lbm_status lbm_load_state(lbm_ctx* c, const void* host_buf) {
    if (!c || !host_buf) return LBM_EINVAL;
    const char* b = (const char*)host_buf;
    const size_t pb = (size_t)stored_blocks(c->p.storage) * c->P * c->elem, fb = c->N * sizeof(float);
    c->cur = 0;
    c->pc = 0;
    CK(c, cudaMemcpyAsync(c->f[0], b, pb, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->phi[0], b + pb, fb, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->phi[1], b + pb + fb, fb, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memcpy(&c->steps, b + pb + 2 * fb, sizeof(long long));
    long long layout = -1;
    std::memcpy(&layout, b + pb + 2 * fb + sizeof(long long), sizeof(long long));
    if ((layout >= 0) != c->aa) return fail(c, LBM_EINVAL, "state saved with the other storage scheme");
    if (c->aa) {
        c->layout = (int)layout;
        c->sp.aa_layout = c->layout;
    }
    c->fields_set = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    return check_err_word(c);
}

extern "C" long long lbm_steps_taken(const lbm_ctx* c) { return c ? c->steps : -1; }

extern "C" int lbm_launches_per_step(const lbm_ctx* c) {
    if (!c) return 0;
    // in place: the colour-field and collide passes, and the near-contact pass
    if (c->aa) return c->p.A_nc > 0.0 ? 3 : 2;
    // the fused step, and the near-contact pass (which writes the ghost copies) or
    // the ghost fill
    if (c->p.A_nc > 0.0) return 2;
    return 1 + (ghost_cells(c->sp) > 0 ? 1 : 0);
}
