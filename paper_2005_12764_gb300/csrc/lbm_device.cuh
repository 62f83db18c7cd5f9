// lbm_device.cuh -- device-side building blocks of the GB300 colour-gradient LB step.
//
// D3Q19 velocity set, population storage formats, and the per-node pieces of one
// time step (Succi et al., arXiv:2005.12764): pull streaming with halfway
// bounce-back, moments (Eq. 3), near-contact force (Eq. 11), total-population BGK
// with the EDM source (Eqs. 1, 2, 5-9), colour-gradient perturbation and
// recolouring (the published colour-gradient method the paper cites).
// All arithmetic is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 19;

// Velocity set ordered lexicographically in (c_z, c_y, c_x): directions 0-4 have
// c_z = -1, 5-13 have c_z = 0 (9 is the rest velocity), 14-18 have c_z = +1. With
// this order the opposite of direction i is 18 - i.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8 || i == 11 || i == 15) ? -1
         : (i == 3 || i == 7 || i == 10 || i == 13 || i == 17) ? 1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 0 || i == 5 || i == 6 || i == 7 || i == 14) ? -1
         : (i == 4 || i == 11 || i == 12 || i == 13 || i == 18) ? 1 : 0;
}
__host__ __device__ constexpr int cz(int i) { return i <= 4 ? -1 : (i >= 14 ? 1 : 0); }
__host__ __device__ constexpr int opp(int i) { return 18 - i; }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
// Weights of the second-order equilibrium, Eq. (2): 1/3, 1/18, 1/36. The FP32
// constants are the nearest single-precision values whose exact sum
// w_0 + 6 w_f + 12 w_e is 1 (0x3EAAAAAC, 0x3D638E38, 0x3CE38E38 = w_f / 2), so that
// sum_i w_i rho reproduces rho without a systematic per-step mass gain.
__host__ __device__ constexpr float wgt(int i) {
    return csq(i) == 0 ? 0.3333333730697632f : (csq(i) == 1 ? 0.0555555522441864f : 0.0277777761220932f);
}
// Isotropy constants B_i of the perturbation operator: -2/9, 1/54, 1/27.
__host__ __device__ constexpr float bpert(int i) {
    return csq(i) == 0 ? -2.0f / 9.0f : (csq(i) == 1 ? 1.0f / 54.0f : 1.0f / 27.0f);
}
// 1/|c_i| for the recolouring angle (0 for the rest velocity).
__host__ __device__ constexpr float inv_clen(int i) {
    return csq(i) == 0 ? 0.0f : (csq(i) == 1 ? 1.0f : 0.70710678118654752f);
}

// ---------------------------------------------------------------- storage formats
// Populations live in [2 species][19 directions][N nodes] arrays. FP32 stores the
// value; FP16/BF16 store the deviation f - ref rounded to nearest even, with the
// reference ref = w_i rho0 (1 +- phi)/2 (+ red, - blue): the species' share of the
// rest population at the reference density, split by the colour field phi of the
// node that wrote the population (in the step that wrote it). In the bulk of either
// phase the stored deviation is then O(|u|, |rho - rho0|) instead of O(w_i rho0/2),
// so the 11-bit FP16 (8-bit BF16) mantissa is spent on the part that changes.
// Deviation reference of species k (0 red, 1 blue) for a direction whose w_i rho0/2
// is hw, at a node with colour field phi. Encoding and decoding both use this one
// expression (explicit FMAs, no contraction choices), so the reference cancels
// exactly and only the rounding of the stored deviation remains.
__device__ __forceinline__ float dev_ref(float hw, float phi, int k) {
    return k == 0 ? __fmaf_rn(hw, phi, hw) : __fmaf_rn(-hw, phi, hw);
}

// Each format says whether it stores deviations (DEV) and whether it is the reduced
// form below (RED).
struct StoreF32 {
    using T = float;
    static constexpr int kind = 0;
    static constexpr bool DEV = false, RED = false;
    __device__ __forceinline__ static float load(const T* p, size_t i, float) { return __ldg(p + i); }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float) { p[i] = v; }
    __device__ __forceinline__ static float cvt(T v, float) { return v; }
    __device__ __forceinline__ static T enc(float v, float) { return v; }
    // (the reduced forms' members; unused by the full forms)
    static constexpr int AUX_BLOCKS = 0;
    __device__ __forceinline__ static float tot_ref(int, float) { return 0.0f; }
    __device__ __forceinline__ static float coef(const T*, size_t, size_t, int) { return 0.0f; }
};
struct StoreF16 {
    using T = __half;
    static constexpr int kind = 1;
    static constexpr bool DEV = true, RED = false;
    __device__ __forceinline__ static float load(const T* p, size_t i, float ref) {
        return __half2float(__ldg(p + i)) + ref;
    }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float ref) {
        p[i] = __float2half_rn(v - ref);
    }
    __device__ __forceinline__ static float cvt(T v, float ref) { return __half2float(v) + ref; }
    __device__ __forceinline__ static T enc(float v, float ref) { return __float2half_rn(v - ref); }
    // (the reduced forms' members; unused by the full forms)
    static constexpr int AUX_BLOCKS = 0;
    __device__ __forceinline__ static float tot_ref(int, float) { return 0.0f; }
    __device__ __forceinline__ static float coef(const T*, size_t, size_t, int) { return 0.0f; }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr int kind = 2;
    static constexpr bool DEV = true, RED = false;
    __device__ __forceinline__ static float load(const T* p, size_t i, float ref) {
        return __bfloat162float(__ldg(p + i)) + ref;
    }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float ref) {
        p[i] = __float2bfloat16_rn(v - ref);
    }
    __device__ __forceinline__ static float cvt(T v, float ref) { return __bfloat162float(v) + ref; }
    __device__ __forceinline__ static T enc(float v, float ref) { return __float2bfloat16_rn(v - ref); }
    // (the reduced forms' members; unused by the full forms)
    static constexpr int AUX_BLOCKS = 0;
    __device__ __forceinline__ static float tot_ref(int, float) { return 0.0f; }
    __device__ __forceinline__ static float coef(const T*, size_t, size_t, int) { return 0.0f; }
};
// Reduced FP32 form, Q + 5 arrays instead of 2Q. The recoloured post-collision
// populations of a node are, per direction,
//   f^r_i = kappa_r f_i + w_i (c_i . m) / |c_i|,   f^b_i = kappa_b f_i - w_i (c_i . m) / |c_i|,
// with f_i their sum, kappa_k = rho_k / rho and m = beta (rho_r rho_b / rho) n (n the
// unit colour gradient, m = 0 where it is undefined). So the total f_i (arrays
// 0 .. Q-1) and the five numbers kappa_r, kappa_b, m_x, m_y, m_z of the node that
// wrote them (arrays Q .. Q+4) determine both species exactly; the pull rebuilds
// each species from the coefficients of the population's source node. (The five
// arrays hold the node's own coefficients: they are read in place, not streamed.)
constexpr int Q5_AUX = 5;   // kappa_r, kappa_b, m_x, m_y, m_z
struct StoreQ5 {
    using T = float;
    static constexpr int kind = 3;
    static constexpr bool DEV = false, RED = true;
    static constexpr int AUX_BLOCKS = Q5_AUX;   // blocks holding the five coefficients
    __device__ __forceinline__ static float load(const T* p, size_t i, float) { return __ldg(p + i); }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float) { p[i] = v; }
    __device__ __forceinline__ static float cvt(T v, float) { return v; }
    __device__ __forceinline__ static T enc(float v, float) { return v; }
    // reference of the stored total of direction i (rho0_ref = 2 ref_half): none
    __device__ __forceinline__ static float tot_ref(int, float) { return 0.0f; }
    // coefficient k of the node at padded index q (P = elements per block)
    __device__ __forceinline__ static float coef(const T* p, size_t P, size_t q, int k) {
        return __ldg(p + (size_t)(Q + k) * P + q);
    }
    __device__ __forceinline__ static void store_coef(T* p, size_t P, size_t q, int k, float v) {
        p[(size_t)(Q + k) * P + q] = v;
    }
};
// Reduced form with FP16 totals, Q + 10 16-bit arrays: the 19 totals as FP16
// deviations f_i - w_i rho0 from the lattice weights (rounded to nearest even; in both
// phases the total density is close to rho0, so the deviation is O(|u|, |rho - rho0|)),
// and the five coefficients kept exact in FP32, each as two 16-bit arrays (low half,
// then high half of its bits), so that the species masses the coefficients carry are
// not rounded. 58 bytes per node and copy instead of 96 (FP32 reduced form) or 152
// (full FP32).
struct StoreQ5H {
    using T = __half;
    static constexpr int kind = 4;
    static constexpr bool DEV = false, RED = true;
    static constexpr int AUX_BLOCKS = 2 * Q5_AUX;
    __device__ __forceinline__ static float load(const T* p, size_t i, float ref) {
        return __half2float(__ldg(p + i)) + ref;
    }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float ref) {
        p[i] = __float2half_rn(v - ref);
    }
    __device__ __forceinline__ static float cvt(T v, float ref) { return __half2float(v) + ref; }
    __device__ __forceinline__ static T enc(float v, float ref) { return __float2half_rn(v - ref); }
    __device__ __forceinline__ static float tot_ref(int i, float rho0) { return wgt(i) * rho0; }
    __device__ __forceinline__ static float coef(const T* p, size_t P, size_t q, int k) {
        const unsigned lo = __half_as_ushort(__ldg(p + (size_t)(Q + 2 * k) * P + q));
        const unsigned hi = __half_as_ushort(__ldg(p + (size_t)(Q + 2 * k + 1) * P + q));
        return __uint_as_float(lo | (hi << 16));
    }
    __device__ __forceinline__ static void store_coef(T* p, size_t P, size_t q, int k, float v) {
        const unsigned b = __float_as_uint(v);
        p[(size_t)(Q + 2 * k) * P + q] = __ushort_as_half((unsigned short)(b & 0xffffu));
        p[(size_t)(Q + 2 * k + 1) * P + q] = __ushort_as_half((unsigned short)(b >> 16));
    }
};
// Recolouring share w_i (c_i . m) / |c_i| of direction i (0 for the rest direction).
__device__ __forceinline__ float q5_share(int i, float mx, float my, float mz) {
    if (csq(i) == 0) return 0.0f;
    float d = 0.0f;
    if (cx(i)) d = cx(i) > 0 ? mx : -mx;
    if (cy(i)) d += cy(i) > 0 ? my : -my;
    if (cz(i)) d += cz(i) > 0 ? mz : -mz;
    return (wgt(i) * inv_clen(i)) * d;
}

// ---------------------------------------------------------------- parameters
struct StepParams {
    const void* fin;        // populations at the start of the step (post-collision)
    const float* phi_lag;   // colour field of the previous step (near-contact rays)
    float* phi_out;         // colour field of this step
    const float* fx_row;    // [ny] x body force per row: g_x + Kolmogorov profile
    const uint8_t* pin_d2;  // [N] squared distance to the nearest pin, 255 = none; or null
    float* ah;              // [N] near-contact strength A_h of this step (A_nc > 0)
    void* ghost_f;          // populations whose ghost copies the list kernel fills (or null)
    float gy, gz;
    float wall_u6;          // 6 U of sliding y-walls (+U at y = ny-1/2, -U at y = -1/2), or 0
    int model;              // 0: colour gradient; 1: Shan-Chen
    float G_sc;             // Shan-Chen coupling G_C (> 0 repulsive)
    int nx, ny, nz;
    size_t N;               // nodes (fields phi, ah are [N], x fastest)
    // population arrays are padded: ghost columns and rows around the lattice (the
    // interior starts padx columns in, 32 bytes), row pitch a multiple of 32 bytes;
    // one [nz][nyp][pitch] block per species/direction
    int pitch, nyp, padx;
    int ghost_arrays;       // blocks with ghost copies (the streamed ones): 2Q, or Q for the
                            // reduced form, whose coefficient blocks follow them
    size_t plane_p, P;      // pitch * nyp, plane_p * nz
    int wall_y, wall_z;
    int var_tau;            // 0: omega0 everywhere; 1: mixture rule per node
    float omega0;
    float inv_nu_r, inv_nu_b;
    float sigma, beta;
    float A_nc, h_min, h_cut, ah_b3, ah_inv;  // A_h tail: b3 = (h_min/h_cut)^3, inv = 1/(1-b3)
    int nsamp;              // ray samples t = -1, -1/2, ..., h_cut + 2
    float ref_half;         // rho0/2 for FP16/BF16 deviation storage and the FP16 reduced
                            // form (whose totals are stored as f_i - w_i rho0), else 0
    int tiles_x, tiles_y;   // xy tiles of the step kernel
    int zparts;             // part mode: z is cut into this many equal parts, one CTA per
                            // (part, tile)
    int chain;              // chain mode (> 0): this many CTAs; the first band_k * tiles
                            // march one tile each over one of band_k bands of band_h planes,
                            // the others share the planes above equally, each a contiguous
                            // run of (tile, plane) units in column-major tile order
    int band_k, band_h;
    void* fout;             // populations after the step
    int* err;               // device error word: 1 = a bounded wait gave up
    int aa_layout;          // in-place (AA) storage: where the state's populations are
                            // (0 or 1, see aa_slot); -1 for the two-copy storage
    int nc_seg;             // near-contact pass: blocks per z segment of a block column
};

static_assert(sizeof(StepParams) % sizeof(int) == 0, "StepParams is copied as ints");

// One lattice of a batched launch: its tensor maps (load: populations of this step,
// store: populations after it), step parameters, the array the step writes (for
// the ghost fill) and its first CTA / first ghost cell in the batched grids.
struct alignas(64) BatchLattice {
    CUtensorMap in_map;
    CUtensorMap out_map;
    StepParams p;
    void* fout;
    int cta_begin;
    long long ghost_begin;
};

// One lattice of a batched near-contact launch: the tensor map of its lagged colour
// field (and whether the pass may use it), its parameters for the step (lagged field,
// A_h, the populations whose ghost copies the pass writes), and its first block of
// nodes and first ghost-copy task in the launch.
struct alignas(64) NcBatchLattice {
    CUtensorMap lag_map;
    StepParams p;
    long long block_begin;
    long long ghost_begin;
    int tma_ok;
};

// ---------------------------------------------------------------- near-contact force
__device__ __forceinline__ float A_h(const StepParams& p, float h) {
    if (h <= p.h_min) return p.A_nc;
    if (h >= p.h_cut) return 0.0f;
    float a = p.h_min / h;
    return p.A_nc * (a * a * a - p.ah_b3) * p.ah_inv;
}

__device__ __forceinline__ int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}
// Wrap of an index that lies within a few periods of [0, n): no integer division in
// the common case; falls back to a modulo (bounded time) for anything further out.
__device__ __forceinline__ int wrap_near(int a, int n) {
    if (a < -4 * n || a >= 5 * n) return wrapi(a, n);
    while (a < 0) a += n;
    while (a >= n) a -= n;
    return a;
}

// Index of node (x, y, z) in one padded population block (x, y may be ghosts, -2..n+1).
__host__ __device__ __forceinline__ size_t pidx(int pitch, int nyp, int padx, int x, int y, int z) {
    return ((size_t)z * nyp + (y + 2)) * pitch + (x + padx);
}

// ---------------------------------------------------------------- in-place (AA) storage
// One copy of the populations, each slot read and then written by the same node in a
// step. The state between steps (the post-collision populations f*_i(x) of the last
// step) sits in one of two layouts, which alternate:
//  layout 0: f*_i(x) in slot (opp(i), x), the node's own slots, reversed;
//  layout 1: f*_i(x) in slot (i, x + c_i), streamed already, or in slot (opp(i), x)
//            when x + c_i lies beyond a wall (the population comes back to x).
// A step from layout 1 reads a node's post-stream populations f_i(x) from its own
// slots (i, x) (a link from beyond a wall included) and writes f*_i(x) in layout 0; a
// step from layout 0 reads f_i(x) = f*_i(x - c_i) from (opp(i), x - c_i) (from (i, x)
// for a link from beyond a wall) and writes layout 1. Either way every node reads and
// writes exactly the same slots, so nodes never race.
// Node (x, y, z) + c_i: false if it lies beyond a wall; else its wrapped coordinates.
__device__ __forceinline__ bool aa_neighbour(const StepParams& p, int i, int x, int y, int z,
                                             int& xn, int& yn, int& zn) {
    yn = y + cy(i);
    zn = z + cz(i);
    if ((p.wall_y && (yn < 0 || yn >= p.ny)) || (p.wall_z && (zn < 0 || zn >= p.nz))) return false;
    xn = wrap_near(x + cx(i), p.nx);
    yn = wrap_near(yn, p.ny);
    zn = wrap_near(zn, p.nz);
    return true;
}
// Slot (direction block `dir`, padded index) of f*_i of node (x, y, z) in `layout`.
__device__ __forceinline__ size_t aa_slot(const StepParams& p, int layout, int i, int x, int y,
                                          int z, int& dir) {
    if (layout == 1) {
        int xn, yn, zn;
        if (aa_neighbour(p, i, x, y, z, xn, yn, zn)) {
            dir = i;
            return pidx(p.pitch, p.nyp, p.padx, xn, yn, zn);
        }
    }
    dir = opp(i);
    return pidx(p.pitch, p.nyp, p.padx, x, y, z);
}

// One term 3 w_i c_i v of the isotropic colour gradient (3 w_i = 1/6 for faces, 1/12
// for edges), accumulated with explicit FMAs in direction order: every kernel that
// evaluates a node's gradient gets the same bits.
__device__ __forceinline__ void grad_add(int i, float v, float& Gx, float& Gy, float& Gz) {
    const float w3 = csq(i) == 1 ? (1.0f / 6.0f) : (1.0f / 12.0f);
    if (cx(i)) Gx = __fmaf_rn(cx(i) > 0 ? w3 : -w3, v, Gx);
    if (cy(i)) Gy = __fmaf_rn(cy(i) > 0 ? w3 : -w3, v, Gy);
    if (cz(i)) Gz = __fmaf_rn(cz(i) > 0 ? w3 : -w3, v, Gz);
}

// Isotropic colour gradient of a node field at (x, y, z); a neighbour beyond a wall
// takes the centre value.
__device__ __forceinline__ void gradient_global(const StepParams& p, const float* phi, int x, int y,
                                                int z, float& Gx, float& Gy, float& Gz) {
    const size_t self = ((size_t)z * p.ny + y) * p.nx + x;
    const float phic = __ldg(phi + self);
    Gx = Gy = Gz = 0.0f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (i == 9) continue;
        const int yy = y + cy(i), zz = z + cz(i);
        const bool wall = (p.wall_y && (yy < 0 || yy >= p.ny)) || (p.wall_z && (zz < 0 || zz >= p.nz));
        float v = phic;
        if (!wall)
            v = __ldg(phi + ((size_t)wrap_near(zz, p.nz) * p.ny + wrap_near(yy, p.ny)) * p.nx +
                      wrap_near(x + cx(i), p.nx));
        grad_add(i, v, Gx, Gy, Gz);
    }
}

// Near-contact strength A_h[h] at a node (Eq. 11, F = A_h[h] G with G the current
// colour gradient). The film is measured on the colour field of the previous step:
// with G' its gradient at the node (|G'| >= 1e-3, else 0) the ray runs along
// n' = -G'/|G'|, sampled every half lattice unit from t = -1 to h_cut + 2. Samples
// within 1e-5 of zero carry no sign; h is the distance between the first downward
// zero crossing and the next upward one, each located by linear interpolation
// between consecutive signed samples; a ray that leaves the fluid through a wall
// stops there. Pinning sites add A_h[d], d the distance to the nearest pin.
constexpr float kSignBand = 1e-5f;

// Ray of a node: unit direction -G'/|G'|; false when |G'| < 1e-3 or non-finite.
__device__ __forceinline__ bool nc_ray(float Gx, float Gy, float Gz, float& nx_, float& ny_,
                                       float& nz_) {
    const float gm = sqrtf(Gx * Gx + Gy * Gy + Gz * Gz);
    if (!(gm >= 1e-3f) || !isfinite(gm)) return false;
    const float inv = 1.0f / gm;
    nx_ = -Gx * inv;
    ny_ = -Gy * inv;
    nz_ = -Gz * inv;
    return true;
}

// First sample of a ray outside the fluid (p.nsamp if none).
__device__ __forceinline__ int nc_sample_end(const StepParams& p, int y, int z, float ny_,
                                             float nz_) {
    int s_end = p.nsamp;
    if (p.wall_y || p.wall_z) {
        const float ylo = (float)-y, yhi = (float)(p.ny - 1 - y);
        const float zlo = (float)-z, zhi = (float)(p.nz - 1 - z);
        auto inside = [&](int s) {
            const float t = -1.0f + 0.5f * (float)s;
            const float oy = t * ny_, oz = t * nz_;
            return !((p.wall_y && !(oy >= ylo && oy <= yhi)) || (p.wall_z && !(oz >= zlo && oz <= zhi)));
        };
        // the samples inside the fluid along a walled axis are one interval of s (t n
        // is monotone in s); if it holds s = 0, it ends near the sample where the ray
        // reaches the wall, estimated and then settled with the exact test
        if (!inside(0)) {
            s_end = 0;
        } else {
            float smax = (float)(p.nsamp - 1);
            if (p.wall_y && ny_ != 0.0f)
                smax = fminf(smax, floorf(2.0f * ((ny_ > 0.0f ? yhi : ylo) / ny_ + 1.0f)));
            if (p.wall_z && nz_ != 0.0f)
                smax = fminf(smax, floorf(2.0f * ((nz_ > 0.0f ? zhi : zlo) / nz_ + 1.0f)));
            int s = max(0, (int)smax);
            while (s + 1 < p.nsamp && inside(s + 1)) ++s;
            while (s > 0 && !inside(s)) --s;
            s_end = s + 1;
        }
    }
    return s_end;
}

// Linear interpolation (1 - w) a + w b with every rounding fixed (no contraction left
// to the compiler), so that a ray sample has the same value however it is evaluated.
__device__ __forceinline__ float ray_lerp(float a, float b, float w) {
    return __fmaf_rn(w, b, __fmul_rn(1.0f - w, a));   // (1 - w) a + w b
}

// Crossing search along one ray, fed its samples in order (t = -1, -1/2, ...):
// feed() returns true once A_h is decided (in `a`); a ray whose samples run out
// first has A_h = 0.
struct NcMarch {
    float t_a = 0.0f, v_a = 0.0f, t_d = 0.0f;
    bool have_a = false, have_d = false;
    __device__ __forceinline__ bool feed(const StepParams& p, float t, float vs, float& a) {
        if (fabsf(vs) <= kSignBand) return false;
        if (have_a) {
            if (!have_d && v_a > 0.0f && vs < 0.0f) {
                t_d = t_a + (t - t_a) * v_a / (v_a - vs);
                have_d = true;
            } else if (have_d && v_a < 0.0f && vs > 0.0f) {
                const float t_u = t_a + (t - t_a) * v_a / (v_a - vs);
                a = A_h(p, t_u - t_d);
                return true;
            }
        }
        // any upward crossing after this sample gives h >= h_cut, where A_h vanishes
        if (have_d && t - t_d >= p.h_cut) {
            a = 0.0f;
            return true;
        }
        t_a = t;
        v_a = vs;
        have_a = true;
        return false;
    }
};

// ---------------------------------------------------------------- collision
// Pairwise (fixed-tree) sum of 19 values; every caller sums the same node's
// populations in the same order, so a node's density is bitwise the same whichever
// thread computes it.
__device__ __forceinline__ float sum19(const float (&v)[Q]) {
    float a = (v[0] + v[1]) + (v[2] + v[3]);
    float b = (v[4] + v[5]) + (v[6] + v[7]);
    float c = (v[8] + v[9]) + (v[10] + v[11]);
    float d = (v[12] + v[13]) + (v[14] + v[15]);
    float e = (v[16] + v[17]) + v[18];
    return ((a + b) + (c + d)) + e;
}

// Colour field (rho_r - rho_b)/(rho_r + rho_b); every thread that evaluates a node's
// colour uses this same expression, so it is bitwise the same wherever computed.
__device__ __forceinline__ float colour(float rr, float rb) {
    return (rr - rb) * __frcp_rn(rr + rb);
}

// Threshold below which the colour gradient is treated as zero (no perturbation,
// no recolouring segregation): above the rounding level (~1e-7) of the FP32
// stencil on an O(1) colour field, so FP32 and FP64 evaluations agree on the branch.
constexpr float kGradZero = 1e-6f;

// Collision of one node from its post-stream total populations f[19], species
// densities and colour gradient; writes the two new species populations through
// the storage format. Order: BGK + EDM source (Eqs. 1, 2, 9) on the total
// population, perturbation Delta_i = (A/2)|G|[w_i (c_i.G)^2/|G|^2 - B_i] with
// A = 9 omega sigma / 2, recolouring f^r = (rho_r/rho) f + beta (rho_r rho_b/rho)
// w_i cos(theta_i), f^b = (rho_b/rho) f - (same).
// Evaluated in "small-number" form: with f'_i = w_i rho + s_i, the outputs are
// f^r_i = w_i rho_r + (rho_r/rho) s_i + seg_i, so the large parts w_i rho_k are
// rounded once and all other terms are O(|u|, |F|, |G|) corrections. Opposite
// directions share their symmetric terms. The rest direction takes minus the sum of
// the other perturbations, so the perturbation conserves mass exactly.
// Output of the collision: one value per direction block k (species * 19 + direction)
// handed to an emitter functor, emit(k, value, ref), with k a compile-time constant
// after unrolling. The emitter writes the plane's shared-memory output tile, which
// the step kernel stores to global memory with tensor copies.
template <class St, int NT>
struct SmemEmit {
    typename St::T* tile;        // this node in block 0 of the shared output tile
    __device__ __forceinline__ void operator()(int k, float v, float ref) const {
        tile[k * NT] = St::enc(v, ref);   // NT nodes per block of the tile
    }
    // reduced forms: recolouring coefficient k (its block(s) after the Q totals)
    __device__ __forceinline__ void coef(int k, float v) const {
        if constexpr (St::RED) {
            if constexpr (St::AUX_BLOCKS == Q5_AUX) {
                tile[(Q + k) * NT] = v;
            } else {
                const unsigned b = __float_as_uint(v);
                tile[(Q + 2 * k) * NT] = __ushort_as_half((unsigned short)(b & 0xffffu));
                tile[(Q + 2 * k + 1) * NT] = __ushort_as_half((unsigned short)(b >> 16));
            }
        }
    }
};

// Momentum j = sum_i c_i f_i of the total populations, summed in one fixed order
// (the collision and the unit-rate march, which carries only the moments, get the
// same bits).
__device__ __forceinline__ void cg_momentum(const float (&f)[Q], float& jx, float& jy, float& jz) {
    jx = 0.f;
    jy = 0.f;
    jz = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float d = f[i] - f[opp(i)];
        if (cx(i)) jx += cx(i) > 0 ? d : -d;
        if (cy(i)) jy += cy(i) > 0 ? d : -d;
        if (cz(i)) jz += cz(i) > 0 ? d : -d;
    }
}

template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void collide_moments(const StepParams& p, const float (&f)[Q], float rr,
                                                float rb, float jx, float jy, float jz, float phi,
                                                float Gx, float Gy, float Gz, float Fx, float Fy,
                                                float Fz, const Emit& emit);

template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void collide_store(const StepParams& p, const float (&f)[Q], float rr,
                                              float rb, float phi, float Gx, float Gy, float Gz,
                                              float Fx, float Fy, float Fz, const Emit& emit) {
    float jx, jy, jz;
    cg_momentum(f, jx, jy, jz);
    collide_moments<St, UnitOmega>(p, f, rr, rb, jx, jy, jz, phi, Gx, Gy, Gz, Fx, Fy, Fz, emit);
}

// The collision from the node's densities and momentum; the total populations f enter
// only the non-equilibrium part, which vanishes at unit rate (omega = 1): there the
// caller may pass any array.
template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void collide_moments(const StepParams& p, const float (&f)[Q], float rr,
                                                float rb, float jx, float jy, float jz, float phi,
                                                float Gx, float Gy, float Gz, float Fx, float Fy,
                                                float Fz, const Emit& emit) {
    const float rho = rr + rb;
    const float inv_rho = __frcp_rn(rho);
    const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    float omega = p.omega0;
    if (!UnitOmega && p.var_tau) {
        const float inv_nu = (rr * p.inv_nu_r + rb * p.inv_nu_b) * inv_rho;
        omega = 1.0f / (3.0f / inv_nu + 0.5f);
    }
    const float om1 = UnitOmega ? 0.0f : 1.0f - omega;
    // BGK + EDM source: f' = f^eq(rho, U) + (1 - omega)(f - f^eq(rho, u)) with the
    // shifted velocity U = u + F/rho, since the source f^eq(U) - f^eq(u) and the
    // relaxed part omega f^eq(u) + (1 - omega) f combine to that (Eqs. 1, 9)
    const float Ux = ux + Fx * inv_rho, Uy = uy + Fy * inv_rho, Uz = uz + Fz * inv_rho;
    const float U15 = 1.5f * (Ux * Ux + Uy * Uy + Uz * Uz);
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float g2 = Gx * Gx + Gy * Gy + Gz * Gz;
    const bool has_g = g2 >= kGradZero * kGradZero;
    const float inv_g = has_g ? rsqrtf(g2) : 0.0f;
    const float gm = g2 * inv_g;
    const float half_A_g = has_g ? 0.5f * (4.5f * omega * p.sigma) * gm : 0.0f;
    const float seg0 = has_g ? p.beta * rr * rb * inv_rho : 0.0f;
    const float ar = rr * inv_rho, ab = rb * inv_rho;
    // deviation references of this node (phi = its colour field of this step); they
    // vanish for FP32 storage, whose store ignores them
    const float refh = p.ref_half;
    // per weight class (face / edge): products that do not depend on the direction
    const float wr_f = wgt(2) * rho, wr_e = wgt(0) * rho;
    const float wrr_f = wgt(2) * rr, wrr_e = wgt(0) * rr;
    const float wrb_f = wgt(2) * rb, wrb_e = wgt(0) * rb;
    const float hw_f = half_A_g * wgt(2), hw_e = half_A_g * wgt(0);
    const float hb_f = half_A_g * bpert(2), hb_e = half_A_g * bpert(0);
    const float sg_f = seg0 * wgt(2) * inv_clen(2), sg_e = seg0 * wgt(0) * inv_clen(0);
    float pert_sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int o = opp(i);
        const bool face = csq(i) == 1;
        const float wr = face ? wr_f : wr_e;
        // f^eq(U) - w rho = e_sym +- e_asym for the pair (i, opposite)
        const float v = (float)cx(i) * Ux + (float)cy(i) * Uy + (float)cz(i) * Uz;
        const float es = wr * (4.5f * v * v - U15);
        const float ea = wr * (3.0f * v);
        const float cg = (float)cx(i) * Gx + (float)cy(i) * Gy + (float)cz(i) * Gz;
        const float cn = cg * inv_g;
        const float dlt = (face ? hw_f : hw_e) * (cn * cn) - (face ? hb_f : hb_e);
        pert_sum += dlt;
        float si = (es + ea) + dlt;
        float so = (es - ea) + dlt;
        if (!UnitOmega) {
            const float a = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
            const float qs = wr * (4.5f * a * a - usq15), qa = wr * (3.0f * a);
            si += om1 * ((f[i] - wr) - (qs + qa));
            so += om1 * ((f[o] - wr) - (qs - qa));
        }
        if constexpr (St::RED) {
            // reduced form: the total; the species split goes with the coefficients
            emit(i, wr + si, St::tot_ref(i, 2.0f * refh));
            emit(o, wr + so, St::tot_ref(o, 2.0f * refh));
        } else {
            const float sg = (face ? sg_f : sg_e) * cn;
            const float wrr = face ? wrr_f : wrr_e, wrb = face ? wrb_f : wrb_e;
            const float hw = wgt(i) * refh;
            const float rf_r = dev_ref(hw, phi, 0), rf_b = dev_ref(hw, phi, 1);
            emit(i, wrr + (ar * si + sg), rf_r);
            emit(o, wrr + (ar * so - sg), rf_r);
            emit(Q + i, wrb + (ab * si - sg), rf_b);
            emit(Q + o, wrb + (ab * so + sg), rf_b);
        }
    }
    {
        constexpr int i = 9;
        const float w = wgt(i);
        const float wr = w * rho;
        float si = -wr * U15 - 2.0f * pert_sum;
        if (!UnitOmega) si += om1 * ((f[i] - wr) + wr * usq15);
        if constexpr (St::RED) {
            emit(i, wr + si, St::tot_ref(i, 2.0f * refh));
        } else {
            const float hw = w * refh;
            emit(i, w * rr + ar * si, dev_ref(hw, phi, 0));
            emit(Q + i, w * rb + ab * si, dev_ref(hw, phi, 1));
        }
    }
    if constexpr (St::RED) {
        // recolouring coefficients: kappa_r, kappa_b and m = seg0 G / |G| (the
        // recolouring term of direction i is then w_i (c_i . m) / |c_i|)
        const float mg = seg0 * inv_g;
        emit.coef(0, ar);
        emit.coef(1, ab);
        emit.coef(2, mg * Gx);
        emit.coef(3, mg * Gy);
        emit.coef(4, mg * Gz);
    }
}

// Shan-Chen collision of one node (the binary mixture of Eqs. (5)-(9), (12)) from
// its post-stream species populations fr, fb, densities rr, rb, colour field phi
// (for deviation storage), cohesive velocity shifts s_k = F^k/rho_k and body force
// F: each species relaxes at the mixture rate towards f^eq(rho_k, u), u = j / rho,
// and takes the EDM source of its own force F^k + (rho_k/rho) F:
//   f^k'_i = f^eq_i(rho_k, U_k) + (1 - omega)(f^k_i - f^eq_i(rho_k, u)),
//   U_k = u + s_k + F / rho.
// Small-number form as in collide_store: f^eq_i(rho_k, U) = w_i rho_k +
// w_i rho_k (3 c.U + 4.5 (c.U)^2 - 1.5 U^2), opposite directions sharing terms.
template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void sc_collide_moments(const StepParams& p, const float (&fr)[Q],
                                                   const float (&fb)[Q], float rr, float rb,
                                                   float jx, float jy, float jz, float phi,
                                                   const float (&sr)[3], const float (&sb)[3],
                                                   float Fx, float Fy, float Fz,
                                                   const Emit& emit);

// Momentum j = sum_i c_i (f^r_i + f^b_i) of the two species' populations, summed in one
// fixed order (the collision and the moments-only march of the unit-rate case get
// the same bits).
__device__ __forceinline__ void sc_momentum(const float (&fr)[Q], const float (&fb)[Q], float& jx,
                                            float& jy, float& jz) {
    jx = 0.f;
    jy = 0.f;
    jz = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float d = (fr[i] + fb[i]) - (fr[opp(i)] + fb[opp(i)]);
        if (cx(i)) jx += cx(i) > 0 ? d : -d;
        if (cy(i)) jy += cy(i) > 0 ? d : -d;
        if (cz(i)) jz += cz(i) > 0 ? d : -d;
    }
}

template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void sc_collide_store(const StepParams& p, const float (&fr)[Q],
                                                 const float (&fb)[Q], float rr, float rb,
                                                 float phi, const float (&sr)[3],
                                                 const float (&sb)[3], float Fx, float Fy,
                                                 float Fz, const Emit& emit) {
    float jx, jy, jz;
    sc_momentum(fr, fb, jx, jy, jz);
    sc_collide_moments<St, UnitOmega>(p, fr, fb, rr, rb, jx, jy, jz, phi, sr, sb, Fx, Fy, Fz,
                                      emit);
}

// The collision from the node's densities and momentum; the populations fr, fb enter
// only the non-equilibrium part, which vanishes at unit rate (omega = 1): there the
// caller may pass any arrays.
template <class St, bool UnitOmega, class Emit>
__device__ __forceinline__ void sc_collide_moments(const StepParams& p, const float (&fr)[Q],
                                                   const float (&fb)[Q], float rr, float rb,
                                                   float jx, float jy, float jz, float phi,
                                                   const float (&sr)[3], const float (&sb)[3],
                                                   float Fx, float Fy, float Fz,
                                                   const Emit& emit) {
    const float rho = rr + rb;
    const float inv_rho = __frcp_rn(rho);
    const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    float omega = p.omega0;
    if (!UnitOmega && p.var_tau) {
        const float inv_nu = (rr * p.inv_nu_r + rb * p.inv_nu_b) * inv_rho;
        omega = 1.0f / (3.0f / inv_nu + 0.5f);
    }
    const float om1 = UnitOmega ? 0.0f : 1.0f - omega;
    const float bx = Fx * inv_rho, by = Fy * inv_rho, bz = Fz * inv_rho;
    const float Urx = ux + sr[0] + bx, Ury = uy + sr[1] + by, Urz = uz + sr[2] + bz;
    const float Ubx = ux + sb[0] + bx, Uby = uy + sb[1] + by, Ubz = uz + sb[2] + bz;
    const float Ur15 = 1.5f * (Urx * Urx + Ury * Ury + Urz * Urz);
    const float Ub15 = 1.5f * (Ubx * Ubx + Uby * Uby + Ubz * Ubz);
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float refh = p.ref_half;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int o = opp(i);
        const float wrr = wgt(i) * rr, wrb = wgt(i) * rb;
        const float vr = (float)cx(i) * Urx + (float)cy(i) * Ury + (float)cz(i) * Urz;
        const float vb = (float)cx(i) * Ubx + (float)cy(i) * Uby + (float)cz(i) * Ubz;
        const float esr = wrr * (4.5f * vr * vr - Ur15), ear = wrr * (3.0f * vr);
        const float esb = wrb * (4.5f * vb * vb - Ub15), eab = wrb * (3.0f * vb);
        float ri = esr + ear, ro = esr - ear, bi = esb + eab, bo = esb - eab;
        if (!UnitOmega) {
            const float a = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
            const float q = 4.5f * a * a - usq15;
            ri += om1 * ((fr[i] - wrr) - wrr * (q + 3.0f * a));
            ro += om1 * ((fr[o] - wrr) - wrr * (q - 3.0f * a));
            bi += om1 * ((fb[i] - wrb) - wrb * (q + 3.0f * a));
            bo += om1 * ((fb[o] - wrb) - wrb * (q - 3.0f * a));
        }
        const float hw = wgt(i) * refh;
        const float rf_r = dev_ref(hw, phi, 0), rf_b = dev_ref(hw, phi, 1);
        emit(i, wrr + ri, rf_r);
        emit(o, wrr + ro, rf_r);
        emit(Q + i, wrb + bi, rf_b);
        emit(Q + o, wrb + bo, rf_b);
    }
    {
        constexpr int i = 9;
        const float w = wgt(i);
        const float wrr = w * rr, wrb = w * rb;
        float ri = -wrr * Ur15, bi = -wrb * Ub15;
        if (!UnitOmega) {
            ri += om1 * ((fr[i] - wrr) + wrr * usq15);
            bi += om1 * ((fb[i] - wrb) + wrb * usq15);
        }
        const float hw = w * refh;
        emit(i, wrr + ri, dev_ref(hw, phi, 0));
        emit(Q + i, wrb + bi, dev_ref(hw, phi, 1));
    }
}

}  // namespace lbm
