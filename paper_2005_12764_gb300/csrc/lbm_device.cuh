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
struct StoreQ5 {
    using T = float;
    static constexpr int kind = 3;
    static constexpr bool DEV = false, RED = true;
    __device__ __forceinline__ static float load(const T* p, size_t i, float) { return __ldg(p + i); }
    __device__ __forceinline__ static void store(T* p, size_t i, float v, float) { p[i] = v; }
    __device__ __forceinline__ static float cvt(T v, float) { return v; }
    __device__ __forceinline__ static T enc(float v, float) { return v; }
};
constexpr int Q5_AUX = 5;   // kappa_r, kappa_b, m_x, m_y, m_z
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
    int4* cand;             // candidates written by the step kernel: nodes with |G| >= 0.9e-3,
                            // {node, G_x, G_y, G_z} (float bits), G of the step's colour field
    int* cand_count;        // its length (reset before the step kernel)
    const int4* nc_list;    // list the near-contact pass works on (null: scan every node)
    const int* nc_count;
    uint32_t* nc_pos;       // [nbz][nby][nbw] bits: block (bx, by, bz) of the 2x2x2 block grid
                            // may hold a node with phi_lag > kPosBand among nodes 2b .. 2b+2
                            // per axis (bit bx & 31 of word bx >> 5)
    uint32_t* nc_pos_out;   // the same bits for phi_out: cleared by the near-contact pass and
                            // set by the step kernel (null: not kept)
    int* nc_next;           // work counter of the near-contact list kernel (0 on entry)
    int* nc_next_clear;     // counter the list kernel zeroes for the next pass (or null)
    int* cand_clear;        // candidate counter the list kernel zeroes for the step kernel
    void* ghost_f;          // populations whose ghost copies the list kernel fills (or null)
    int nbx, nby, nbz, nbw; // block grid: ceil(n / 2) per axis; nbw = ceil(nbx / 32)
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
    float ref_half;         // rho0/2 for FP16/BF16 deviation storage, 0 for FP32
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
//
// Work bound (exact): an upward crossing needs a positive sample, and a trilinear
// sample is a convex combination of its 8 corner nodes, so it cannot exceed 1e-5
// when every corner is <= kPosBand = 1e-5/2. A bit field over 2x2x2 blocks marks
// where such a corner may be; samples after the last marked one cannot complete a
// crossing pair, so the march ends there with the same A_h. Most candidate rays
// (outward from a droplet into the bulk) have no marked sample at all.
constexpr float kSignBand = 1e-5f;
constexpr float kPosBand = 0.5e-5f;

// Blocks of the bit field that hold node n of an axis of N nodes (nb = ceil(N/2)
// blocks, block b = nodes 2b, 2b+1, 2b+2): `second` = 0 gives n/2, `second` = 1 the
// other block holding it, or -1. Even n >= 2 also lie in block n/2 - 1; on a
// periodic axis the last block wraps over node 0 (and over node 1 when N is odd).
__device__ __forceinline__ int pos_block(int n, int second, int N, bool periodic, int nb) {
    if (!second) return n >> 1;
    if ((n & 1) == 0 && n >= 2) return (n >> 1) - 1;
    if (periodic && (n == 0 || (n == 1 && (N & 1)))) return nb - 1;
    return -1;
}

// Bits 0, 2, .., 30 of v moved to bits 0 .. 15.
__device__ __forceinline__ uint32_t even_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    return (v | (v >> 8)) & 0x0000FFFFu;
}

// Marks, in the bit field `bits`, the blocks holding the positive nodes of one row
// segment: m = bit j set if node (x0 + j, y, z) has phi > kPosBand, x0 even, the
// segment at most 32 nodes. Lane `which` (0 .. 3) of the calling warp handles the
// (y, z) block pair (which & 1, which >> 1). The blocks x0/2 .. x0/2 + 15 take their
// nodes 2b, 2b+1, 2b+2 from the segment (node x0 + 32 belongs to the next segment,
// which marks it as its own first node); the block before the segment (wrapping
// at x = 0) holds node x0, and for odd nx node 1 as well.
__device__ __forceinline__ void mark_pos_row(uint32_t* bits, const StepParams& p, int x0, int y,
                                             int z, uint32_t m, int which) {
    const int by = pos_block(y, which & 1, p.ny, !p.wall_y, p.nby);
    const int bz = pos_block(z, which >> 1, p.nz, !p.wall_z, p.nbz);
    if (by < 0 || bz < 0) return;
    uint32_t* row = bits + ((size_t)bz * p.nby + by) * p.nbw;
    const uint32_t c = even_bits(m | (m >> 1) | (m >> 2));
    const int b0 = x0 >> 1;
    if (c) atomicOr(row + (b0 >> 5), c << (b0 & 31));
    if ((m & 1u) || (x0 == 0 && (p.nx & 1) && (m & 2u))) {
        const int pb = x0 == 0 ? p.nbx - 1 : b0 - 1;
        atomicOr(row + (pb >> 5), 1u << (pb & 31));
    }
}

// Ray of a candidate: unit direction -G'/|G'|; false when |G'| < 1e-3 or non-finite.
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

// Ray sample positions: cell b = base + floor(o) and fraction o - floor(o) along one
// axis, for |o| <= h_cut + 2 <= 11. Periodic axes of at least 12 nodes wrap with one
// conditional add or subtract; shorter ones take the general wrap. On a walled axis
// the point lies inside the fluid iff -base <= o <= n - 1 - base, i.e. its cell is a
// fluid node and it does not pass the last node.
__device__ __forceinline__ int ray_wrap(int b, int n) {
    if (n >= 12) {
        b = b < 0 ? b + n : b;
        return b >= n ? b - n : b;
    }
    return wrap_near(b, n);
}

// Index of the last sample of a ray that may be positive, or -1: the samples
// inside the fluid are s < s_end (the first sample outside stops the march), and
// the bit field is scanned from s_end - 1 downwards. A sample on the last node of
// a walled axis (fraction 0) is looked up in that node's block: its value is that
// node's, whatever the other corner holds. (Starting the march at the first
// possibly positive sample instead of t = -1 gives the same A_h, but finding that
// sample by a forward scan costs more than the samples it saves.)
__device__ __forceinline__ bool nc_sample_marked(const StepParams& p, int x, int y, int z,
                                                 float nx_, float ny_, float nz_, int s) {
    const float t = -1.0f + 0.5f * (float)s;
    const int ix = ray_wrap(x + (int)floorf(t * nx_), p.nx);
    const int iy = ray_wrap(y + (int)floorf(t * ny_), p.ny);   // identity on walled axes
    const int iz = ray_wrap(z + (int)floorf(t * nz_), p.nz);
    const int bx = ix >> 1;
    const uint32_t w = __ldg(p.nc_pos + ((iz >> 1) * p.nby + (iy >> 1)) * p.nbw + (bx >> 5));
    return (w >> (bx & 31)) & 1u;
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

__device__ __forceinline__ int nc_last_sample(const StepParams& p, int x, int y, int z, float nx_,
                                              float ny_, float nz_) {
    const int s_end = nc_sample_end(p, y, z, ny_, nz_);
    for (int s = s_end - 1; s >= 0; --s)
        if (nc_sample_marked(p, x, y, z, nx_, ny_, nz_, s)) return s;
    return -1;
}

// Trilinear sample of the lagged colour field at node (x, y, z) + offset o, for a
// point known to lie inside the fluid (as nc_last_sample established). The cell and
// the weights come from the offset alone (|o| is small), so the point is located to
// the precision of o, not of x + o; on the last node of a walled axis (fraction 0)
// the cell below is used with fraction 1, which gives that node's value.
// Split into the cell (corner indices and fractions), its 8 corner values, and the
// interpolation, so that a ray can keep the corners while it stays in one cell; the
// interpolation fixes every rounding (no contraction left to the compiler), so a
// sample has the same value however it is evaluated.
struct RayCell {
    int r00, r01, r10, r11;   // row offsets of the corners (z0 y0, z0 y1, z1 y0, z1 y1)
    int ix0, ix1;
    float fx, fy, fz;
};
__device__ __forceinline__ void ray_cell(const StepParams& p, int x, int y, int z, float ox,
                                         float oy, float oz, RayCell& c) {
    const float flx = floorf(ox), fly = floorf(oy), flz = floorf(oz);
    c.fx = ox - flx;
    c.fy = oy - fly;
    c.fz = oz - flz;
    int ix0 = x + (int)flx, iy0 = y + (int)fly, iz0 = z + (int)flz;
    int iy1, iz1;
    ix0 = ray_wrap(ix0, p.nx);
    c.ix0 = ix0;
    c.ix1 = ix0 + 1 == p.nx ? 0 : ix0 + 1;
    if (p.wall_y) {
        if (iy0 == p.ny - 1) {
            iy0 = p.ny - 2;
            c.fy = 1.0f;
        }
        iy1 = iy0 + 1;
    } else {
        iy0 = ray_wrap(iy0, p.ny);
        iy1 = iy0 + 1 == p.ny ? 0 : iy0 + 1;
    }
    if (p.wall_z) {
        if (iz0 == p.nz - 1) {
            iz0 = p.nz - 2;
            c.fz = 1.0f;
        }
        iz1 = iz0 + 1;
    } else {
        iz0 = ray_wrap(iz0, p.nz);
        iz1 = iz0 + 1 == p.nz ? 0 : iz0 + 1;
    }
    c.r00 = (iz0 * p.ny + iy0) * p.nx;
    c.r01 = (iz0 * p.ny + iy1) * p.nx;
    c.r10 = (iz1 * p.ny + iy0) * p.nx;
    c.r11 = (iz1 * p.ny + iy1) * p.nx;
}
__device__ __forceinline__ void ray_corners(const StepParams& p, const RayCell& c, float (&v)[8]) {
    const float* f = p.phi_lag;
    v[0] = __ldg(f + c.r00 + c.ix0);
    v[1] = __ldg(f + c.r00 + c.ix1);
    v[2] = __ldg(f + c.r01 + c.ix0);
    v[3] = __ldg(f + c.r01 + c.ix1);
    v[4] = __ldg(f + c.r10 + c.ix0);
    v[5] = __ldg(f + c.r10 + c.ix1);
    v[6] = __ldg(f + c.r11 + c.ix0);
    v[7] = __ldg(f + c.r11 + c.ix1);
}
__device__ __forceinline__ float ray_lerp(float a, float b, float w) {
    return __fmaf_rn(w, b, __fmul_rn(1.0f - w, a));   // (1 - w) a + w b
}
__device__ __forceinline__ float ray_interp(const RayCell& c, const float (&v)[8]) {
    const float c0 = ray_lerp(ray_lerp(v[0], v[1], c.fx), ray_lerp(v[2], v[3], c.fx), c.fy);
    const float c1 = ray_lerp(ray_lerp(v[4], v[5], c.fx), ray_lerp(v[6], v[7], c.fx), c.fy);
    return ray_lerp(c0, c1, c.fz);
}
__device__ __forceinline__ float ray_sample(const StepParams& p, int x, int y, int z, float ox,
                                            float oy, float oz) {
    RayCell c;
    ray_cell(p, x, y, z, ox, oy, oz, c);
    float v[8];
    ray_corners(p, c, v);
    return ray_interp(c, v);
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
            emit(i, wr + si, 0.0f);
            emit(o, wr + so, 0.0f);
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
            emit(i, wr + si, 0.0f);
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
        emit(Q, ar, 0.0f);
        emit(Q + 1, ab, 0.0f);
        emit(Q + 2, mg * Gx, 0.0f);
        emit(Q + 3, mg * Gy, 0.0f);
        emit(Q + 4, mg * Gz, 0.0f);
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
