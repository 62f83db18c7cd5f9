// lbm_step.cu -- the fused time-step kernel (one launch = one full lattice update),
// the ghost-copy fill and the near-contact pass.
//
// Data layout: populations in [2 species][19 directions][z][y][x] (x fastest), two
// copies (read one, write the other). Each [z][y][x] block is padded: the interior
// of a row starts 32 bytes in (the sector holding the two x ghosts before it) and is
// followed by another such sector, and there are two ghost rows on each side; on
// periodic axes the ghosts hold copies of the wrapped-around nodes, written by the
// ghost-copy fill after every step.
//
// A CTA owns a TX x TY tile of (x, y) columns and marches along z over one part of
// the lattice height. For every plane p it stages in shared memory, per species and
// direction i, the (TX + 16 bytes of halo on each side) x (TY+2) box of the source
// plane p - c_iz that the pull of the tile and of a one-node ring around it reads
// (columns x0-2 .. x0+TX+1, rows y0-1-c_iy .. y0+TY-c_iy): 38 TMA tensor copies, one
// per issuing thread, completing on an mbarrier. The copy of plane p+2 is issued as
// soon as every thread has pulled plane p+1, so it overlaps the collision of plane
// p; two CTAs share an SM, so one CTA's pulls overlap the other's collisions. From a
// staged plane every thread pulls its node with constant-offset shared-memory loads,
// the colour field of the plane (tile + ring) goes to a 4-slot ring buffer, and one
// plane behind, the owned nodes are collided using the isotropic gradient read from
// that ring. The colour field of the same step is thus available at all 18
// neighbours without a second pass over the populations. Links whose source lies
// beyond a bounce-back wall read the node's own opposite population directly from
// global memory. The collision writes the plane's outputs to a shared output tile
// that one thread stores with 38 TMA tensor copies.
//
// Reduced form (Q + 5 blocks: the 19 total populations, then the five recolouring
// coefficients of the node that wrote them): only the totals are staged by tensor
// copies; the coefficients of the (TX+4) x (TY+4) source columns of each plane go to
// a 4-slot ring with plain loads, and each pulled total is split into the two
// species with the coefficients of its source node. The output tile has Q + 5
// blocks.
//
// Work split, two modes.
// Part mode (lattices of more tiles than the GPU holds CTAs at once): z is cut into
// `zparts` equal parts and every CTA marches one part of one tile. CTAs are numbered
// part-major, so the CTAs resident at the same time work on neighbouring tiles at
// the same heights: the halo rows one tile stages are the rows its neighbours are
// reading, and come from L2 rather than HBM.
// Chain mode (smaller lattices): as many CTAs as fit on the GPU at once, each with
// the same number of (tile, plane) units. The lattice height is cut into band_k
// bands of band_h planes, one CTA per (band, tile), and the planes above them,
// whose units the remaining CTAs share in contiguous runs (column-major tile order,
// so such a CTA may finish one tile and continue on the next). Every SM then
// carries the same work, where whole parts per tile would leave some SMs with one
// CTA and others with two; within a band every tile is marched at the same heights
// at the same time, so the halo rows neighbours read come from L2.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <utility>

#include "lbm_device.cuh"

namespace lbm {

constexpr int TX = 32, TY = 8, NT = TX * TY;
static_assert(TX == 32, "a warp is one row of a tile (near-contact bits, row stores)");
constexpr int CTAS_PER_SM = 2;
constexpr int SH = TY + 2, SWP = TX + 2;   // staged rows; colour-field ring columns
constexpr int NRING = 2 * (TX + 2) + 2 * TY;
// Threads that issue a plane's tensor copies, one copy each: the loads from thread
// LOAD_T0 on, the stores from STORE_T0 on, in warps that pull no ring node (threads
// 0 .. NRING-1 do), so that the issue is spread and off the busiest warps.
constexpr int LOAD_T0 = 96, STORE_T0 = 160;
static_assert(NRING <= LOAD_T0 && LOAD_T0 + 2 * Q <= STORE_T0 && STORE_T0 + 2 * Q <= NT,
              "copy-issuing threads");

template <class St, bool SC = false>
struct Geo {
    using T = typename St::T;
    // interior offset in a padded row: 32 bytes, so that each row's two x ghosts
    // (just before the interior, and just after it) sit in 32-byte sectors of their
    // own, written whole by the ghost fill; tile stores start on a 16-byte boundary
    static constexpr int PADX = 32 / (int)sizeof(T);
    // load box: columns x0-HALO .. x0+TX+HALO-1 (covers the pulls x0-2 .. x0+TX+1)
    static constexpr int HALO = 16 / (int)sizeof(T);
    static constexpr int BW = TX + 2 * HALO;
    static constexpr int BOX_BYTES = BW * SH * (int)sizeof(T);
    static constexpr int IK_BYTES = (BOX_BYTES + 127) / 128 * 128;   // 128-byte aligned boxes
    static constexpr int IKS = IK_BYTES / (int)sizeof(T);             // elements per box slot
    // streamed blocks (staged per plane) and stored blocks (output tile): 2Q, or for
    // the reduced form the Q totals and Q + 5 with the recolouring coefficients
    static constexpr bool RED = St::RED;
    static constexpr int NL = RED ? Q : 2 * Q;
    static constexpr int NS = RED ? Q + St::AUX_BLOCKS : 2 * Q;
    static constexpr size_t STAGE_BYTES = (size_t)NL * IK_BYTES;
    // 4-slot ring per plane (tile + ring nodes): the colour field, or for the
    // Shan-Chen model the two species densities
    static constexpr size_t PHI_BYTES = (SC ? 2 : 1) * 4 * SH * SWP * sizeof(float);
    // deviation storage: 4-slot ring of the lagged colour field, (TX+4) x (TY+4) per
    // plane (the sources of the tile and its ring), which decodes the pulled values
    // reduced form: the same ring holds the five recolouring coefficients of every
    // source node, [slot][5][TY+4][TX+4]
    static constexpr bool DEV = St::DEV;
    static constexpr int LW = TX + 4, LH = TY + 4;
    static constexpr size_t LAG_BYTES = DEV ? 4 * LH * LW * sizeof(float)
                                        : (RED ? 4 * Q5_AUX * LH * LW * sizeof(float) : 0);
    // output tile of a plane, [NS][TY][TX], stored by tensor copies
    static constexpr size_t OUT_BYTES = (size_t)NS * TX * TY * sizeof(T);
    static constexpr int STAGES = 1;   // staged planes per CTA
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + OUT_BYTES + PHI_BYTES + LAG_BYTES +
                                   2 * sizeof(unsigned long long);
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}
// Tensor store of one box from shared memory (bulk group), and the group waits.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                             const void* src) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (2^24 by default),
// records the failure in the error word and returns false (the caller then stops).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int* err,
                                          uint32_t limit = 1u << 24) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
}

// Self-test of the bounded wait: an mbarrier that expects one arrival nobody makes.
// The wait gives up after `limit` polls and sets the error word; nothing faults,
// traps or hangs, and the context stays usable.
__global__ void wait_timeout_kernel(int* err, uint32_t limit) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0u, err, limit);
}

cudaError_t launch_wait_selftest(int* err, cudaStream_t s) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(err, 1u << 16);
    return cudaGetLastError();
}

// Programmatic dependent launch: kernels of the time step are launched so that the
// next one may be scheduled while the previous one drains; each waits for the
// previous kernel's completion (and its memory) at grid_dep_wait() before it reads
// or writes any global data, and lets the next one be scheduled at
// grid_dep_launch(). Both are no-ops in a plain launch.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- the kernel
// Body of the step kernel for CTA `cta` of one lattice's grid: the single-lattice
// kernel passes its parameters and tensor maps (kernel parameter space), the
// batched kernel those of the lattice the CTA belongs to.
template <class St, bool UnitOmega, bool SC = false>
__device__ __forceinline__ void step_body(const StepParams& p, const CUtensorMap* fin_map,
                                          const CUtensorMap* fout_map, const int cta) {
    using T = typename St::T;
    using G = Geo<St, SC>;
    constexpr int BW = G::BW, IKS = G::IKS, PADX = G::PADX, HALO = G::HALO, STAGES = G::STAGES;
    static_assert(!(SC && St::RED), "the reduced form holds recoloured populations only");
    // a ring of source-node data per plane: the lagged colour field (deviation
    // storage) or the recolouring coefficients (reduced form)
    constexpr bool RING = G::DEV || G::RED;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage0 = reinterpret_cast<T*>(smem);
    T* sout = reinterpret_cast<T*>(smem + STAGES * G::STAGE_BYTES);           // [2Q][TY][TX]
    unsigned char* rest = smem + STAGES * G::STAGE_BYTES + G::OUT_BYTES;
    float* sphi = reinterpret_cast<float*>(rest);                              // [4][SH][SWP]
    float* slag = reinterpret_cast<float*>(rest + G::PHI_BYTES);
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(rest + G::PHI_BYTES + G::LAG_BYTES);

    const T* __restrict__ fin = static_cast<const T*>(p.fin);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const size_t plane = (size_t)p.nx * p.ny;
    // the output block this thread stores per plane (one tensor copy), or -1
    const int my_st = (tid >= STORE_T0 && tid < STORE_T0 + G::NS) ? tid - STORE_T0 : -1;

    if (tid == 0) {
        mbar_init(&bars[0], G::NL);   // one arrival per staged box
        mbar_init(&bars[1], G::NL);
        fence_mbar_init();
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(fin_map)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(fout_map)) : "memory");
    }
    __syncthreads();
    grid_dep_wait();
    uint32_t parity = 0u;   // bit b: phase parity of buffer b's barrier
    bool failed = false;

    // work of this CTA: one or more segments, each a tile and a range of planes
    const int ntiles = p.tiles_x * p.tiles_y;
    // chain mode: CTAs below nfull march one tile over one band of band_h planes;
    // the others share the units (tile, plane) of the planes from zr up
    const int nfull = p.band_k * ntiles, zr = p.band_k * p.band_h, nr = p.nz - zr;
    long long u_next = 0, u_end = 0;   // chain mode: this CTA's units above zr
    if (p.chain > 0 && cta >= nfull) {
        const long long U = (long long)ntiles * nr;
        const long long R = p.chain - nfull;
        u_next = U * (cta - nfull) / R;
        u_end = U * (cta - nfull + 1) / R;
    }
    bool part_done = false;
    auto next_segment = [&](int& sx0, int& sy0, int& szb, int& sze) -> bool {
        if (p.chain > 0 && cta < nfull) {
            // one band of one tile; consecutive CTAs are neighbours along x, and a
            // band's CTAs all march at the same heights
            if (part_done) return false;
            part_done = true;
            const int band = cta / ntiles, tile = cta - band * ntiles;
            szb = band * p.band_h;
            sze = szb + p.band_h;
            sx0 = (tile % p.tiles_x) * TX;
            sy0 = (tile / p.tiles_x) * TY;
            return true;
        }
        if (p.chain > 0) {
            // units in column-major tile order: tile t is column t / tiles_y, row
            // t % tiles_y; planes zr .. nz-1 ascending within a tile
            if (u_next >= u_end) return false;
            const int t = (int)(u_next / nr);
            szb = zr + (int)(u_next - (long long)t * nr);
            sze = (int)min((long long)p.nz, (long long)szb + (u_end - u_next));
            u_next += sze - szb;
            const int tx = t / p.tiles_y;
            sx0 = tx * TX;
            sy0 = (t - tx * p.tiles_y) * TY;
            return true;
        }
        // part mode: one (z part, tile) item per CTA, part-major
        if (part_done) return false;
        part_done = true;
        const int part = cta / ntiles, tile = cta - part * ntiles;
        szb = (int)((long long)p.nz * part / p.zparts);
        sze = (int)((long long)p.nz * (part + 1) / p.zparts);
        sx0 = (tile % p.tiles_x) * TX;
        sy0 = (tile / p.tiles_x) * TY;
        return true;
    };
    int seg_x0 = 0, seg_y0 = 0, seg_zb = 0, seg_ze = 0;
    while (!failed && next_segment(seg_x0, seg_y0, seg_zb, seg_ze)) {
        const int zb = seg_zb, ze = seg_ze, x0 = seg_x0, y0 = seg_y0;
        const int xw = min(TX, p.nx - x0), yh = min(TY, p.ny - y0);   // owned extent

        // ---- this thread's owned node and (optionally) one ring node
        const int otx = tid % TX, oty = tid / TX;
        const bool owned = otx < xw && oty < yh;
        int rtx = 0, rty = 0;
        bool ring = false;
        if (tid < NRING) {
            if (tid < TX + 2) { rtx = tid - 1; rty = -1; }
            else if (tid < 2 * (TX + 2)) { rtx = tid - (TX + 2) - 1; rty = yh; }
            else if (tid < 2 * (TX + 2) + TY) { rtx = -1; rty = tid - 2 * (TX + 2); }
            else { rtx = xw; rty = tid - 2 * (TX + 2) - TY; }
            ring = rtx <= xw && rty <= yh;
            if (tid >= 2 * (TX + 2) && rty >= yh) ring = false;   // columns cover owned rows
            const int gy = y0 + rty;
            if (p.wall_y && (gy < 0 || gy >= p.ny)) ring = false;  // beyond a wall: unused
        }

        // ---- staging of plane pl into buffer b: one box per species and direction,
        // taken from source plane pl - c_iz
        // threads 0..NL-1 each issue the box of one (species, direction) and arrive on
        // the barrier (with 0 bytes if the box is not needed)
        const int my_ik = (tid >= LOAD_T0 && tid < LOAD_T0 + G::NL) ? tid - LOAD_T0 : -1;
        const int my_i = my_ik < Q ? my_ik : my_ik - Q;
        const int my_cy = my_ik >= 0 ? cy(my_i) : 0, my_cz = my_ik >= 0 ? cz(my_i) : 0;
        auto issue = [&](int b, int pl) {
            if (my_ik < 0) return;
            T* st = stage0 + (size_t)b * (G::NL * IKS);
            const int zs0 = pl - my_cz;
            const bool need = !failed && (!p.wall_z || (pl >= 0 && pl < p.nz)) &&
                              !(p.wall_z && (zs0 < 0 || zs0 >= p.nz));
            if (need) {
                // box origin: interior x0 - HALO and y0 - 1 - c_iy, in padded coordinates
                mbar_arrive_tx(&bars[b], (uint32_t)G::BOX_BYTES);
                tma_load_4d(st + (size_t)my_ik * IKS, fin_map, x0 + PADX - HALO, y0 + 1 - my_cy,
                            wrap_near(zs0, p.nz), my_ik, &bars[b]);
            } else {
                mbar_arrive_tx(&bars[b], 0u);
            }
        };
        auto wait = [&](int b) {
            if (!failed && !mbar_wait(&bars[b], (parity >> b) & 1u, p.err)) failed = true;
            parity ^= 1u << b;
        };

        // lagged colour field of column (tx, ty) (tile coordinates, -2 .. TX+1 and
        // -2 .. TY+1) in lag-ring slot sl
        auto lag_at = [&](int sl, int tx, int ty) -> float& {
            return slag[(sl * G::LH + ty + 2) * G::LW + tx + 2];
        };
        // reduced form: the recolouring coefficients of source column (tx, ty) in ring
        // slot sl; a slot holds the pairs (kappa_r, kappa_b) [LN] (one 8-byte load),
        // then m_x, m_y, m_z [LN] each
        constexpr int LN = G::LW * G::LH;
        struct Coef {
            float kr, kb;
            const float* m;   // m_x; m_y, m_z follow at strides of LN
        };
        auto coef_at = [&](int sl, int tx, int ty) -> Coef {
            const float* b = slag + (size_t)sl * (Q5_AUX * LN);
            const int idx = (ty + 2) * G::LW + tx + 2;
            const float2 k = reinterpret_cast<const float2*>(b)[idx];
            return Coef{k.x, k.y, b + 2 * LN + idx};
        };
        // ---- reduced form: pull of the totals of node (tx, ty) of plane pl (wrapped; sc
        // = ring slot of the unwrapped plane) from staged buffer b, and the species
        // densities rebuilt from the coefficients of each population's source node: the
        // node x - c_i, or for a link bounced back at a wall the node itself, whose
        // population of the opposite direction carries the opposite share
        auto pull_red = [&](int b, int pl, int sc, int tx, int ty, float (&ft)[Q], float& rr,
                            float& rb) {
            const T* st = stage0 + (size_t)b * (G::NL * IKS) + (size_t)(ty + 1) * BW + (tx + HALO);
            const int gy = y0 + ty;
            const bool ylo = p.wall_y && gy == 0, yhi = p.wall_y && gy == p.ny - 1;
            const bool zlo = p.wall_z && pl == 0, zhi = p.wall_z && pl == p.nz - 1;
            const float rho0 = 2.0f * p.ref_half;   // reference of the stored totals
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = St::cvt(st[(size_t)i * IKS - cx(i)], St::tot_ref(i, rho0));
            float sr = 0.f, sb = 0.f, d = 0.f;
            if (!(ylo || yhi || zlo || zhi)) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const Coef a = coef_at((sc - cz(i)) & 3, tx - cx(i), ty - cy(i));
                    sr = __fmaf_rn(a.kr, ft[i], sr);
                    sb = __fmaf_rn(a.kb, ft[i], sb);
                    d += q5_share(i, a.m[0], a.m[LN], a.m[2 * LN]);
                }
            } else {
                const size_t self = pidx(p.pitch, p.nyp, PADX, wrap_near(x0 + tx, p.nx), gy, pl);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const bool out = (cy(i) > 0 && ylo) || (cy(i) < 0 && yhi) ||
                                     (cz(i) > 0 && zlo) || (cz(i) < 0 && zhi);
                    if (out) ft[i] = St::load(fin, (size_t)opp(i) * p.P + self, St::tot_ref(opp(i), rho0));
                    const Coef a = out ? coef_at(sc, tx, ty)
                                       : coef_at((sc - cz(i)) & 3, tx - cx(i), ty - cy(i));
                    sr = __fmaf_rn(a.kr, ft[i], sr);
                    sb = __fmaf_rn(a.kb, ft[i], sb);
                    const float sh = q5_share(i, a.m[0], a.m[LN], a.m[2 * LN]);
                    d += out ? -sh : sh;
                }
            }
            rr = sr + d;
            rb = sb - d;
        };
        // ---- pull of the two species' populations of node (tx, ty) of plane pl
        // (wrapped; sc = lag-ring slot of the unwrapped plane) from staged buffer b, and
        // their densities; wall_terms adds the sliding-wall terms per species.
        auto pull_species = [&](int b, int pl, int sc, int tx, int ty, float (&vr)[Q],
                                float (&vb)[Q], float& rr, float& rb, bool wall_terms) {
            const T* st = stage0 + (size_t)b * (G::NL * IKS) + (size_t)(ty + 1) * BW + (tx + HALO);
            const int gy = y0 + ty;
            const bool ylo = p.wall_y && gy == 0, yhi = p.wall_y && gy == p.ny - 1;
            const bool zlo = p.wall_z && pl == 0, zhi = p.wall_z && pl == p.nz - 1;
            const bool any_wall = ylo || yhi || zlo || zhi;
            const float refh = p.ref_half;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float hw = wgt(i) * refh;
                float rf_r = hw, rf_b = hw;
                if (G::DEV) {
                    const float ph = lag_at((sc - cz(i)) & 3, tx - cx(i), ty - cy(i));
                    rf_r = dev_ref(hw, ph, 0);
                    rf_b = dev_ref(hw, ph, 1);
                }
                vr[i] = St::cvt(st[(size_t)i * IKS - cx(i)], rf_r);
                vb[i] = St::cvt(st[(size_t)(Q + i) * IKS - cx(i)], rf_b);
            }
            if (any_wall) {
                const size_t self = pidx(p.pitch, p.nyp, PADX, wrap_near(x0 + tx, p.nx), gy, pl);
                const float ph_self = G::DEV ? lag_at(sc, tx, ty) : 0.0f;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const bool out = (cy(i) > 0 && ylo) || (cy(i) < 0 && yhi) ||
                                     (cz(i) > 0 && zlo) || (cz(i) < 0 && zhi);
                    if (out) {
                        const float hw = wgt(i) * refh;
                        vr[i] = St::load(fin, (size_t)opp(i) * p.P + self, dev_ref(hw, ph_self, 0));
                        vb[i] = St::load(fin, (size_t)(Q + opp(i)) * p.P + self, dev_ref(hw, ph_self, 1));
                    }
                }
            }
            rr = sum19(vr);
            rb = sum19(vb);
            if (wall_terms && p.wall_u6 != 0.0f && (ylo || yhi)) {
                // sliding y-walls, per species: a link back from a wall moving with
                // (+-U, 0, 0) gains 6 w_i rho_k c_ix (+-U) (these cancel in rho_k)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (cx(i) == 0) continue;
                    const float m = wgt(i) * (float)cx(i) * p.wall_u6;
                    if (cy(i) > 0 && ylo) {
                        vr[i] -= m * rr;
                        vb[i] -= m * rb;
                    }
                    if (cy(i) < 0 && yhi) {
                        vr[i] += m * rr;
                        vb[i] += m * rb;
                    }
                }
            }
        };
        // pull of node (tx, ty) of plane pl (wrapped; sc = lag-ring slot of the
        // unwrapped plane) from staged buffer b; returns densities, and for keep ==
        // true also the total populations. Deviation storage decodes every value
        // against the colour field its source node had when it wrote it.
        auto pull = [&](int b, int pl, int sc, int tx, int ty, float (&ft)[Q], float& rr,
                        float& rb, bool keep) {
            if constexpr (G::RED) {
                pull_red(b, pl, sc, tx, ty, ft, rr, rb);
            } else {
                float vr[Q], vb[Q];
                pull_species(b, pl, sc, tx, ty, vr, vb, rr, rb, false);
                if (keep) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) ft[i] = vr[i] + vb[i];
                }
            }
            if (keep) {
                const int gy = y0 + ty;
                const bool ylo = p.wall_y && gy == 0, yhi = p.wall_y && gy == p.ny - 1;
                if (p.wall_u6 != 0.0f && (ylo || yhi)) {
                    // sliding y-walls: a link back from a wall moving with (+-U, 0, 0)
                    // gains 6 w_i rho c_ix (+-U) (the sum of the two species' shares
                    // rho_k; these terms cancel in the densities)
                    const float rho = rr + rb;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (cx(i) == 0) continue;
                        const float m = wgt(i) * rho * (float)cx(i) * p.wall_u6;
                        if (cy(i) > 0 && ylo) ft[i] -= m;   // from the wall at y = -1/2
                        if (cy(i) < 0 && yhi) ft[i] += m;   // from the wall at y = ny - 1/2
                    }
                }
            }
        };
        auto slot = [](int z) { return (z + 4) & 3; };
        auto phi_at = [&](int s, int tx, int ty) -> float& {
            return sphi[(s * SH + ty + 1) * SWP + tx + 1];
        };
        // colour field of plane pl (tile + ring) from buffer b; owned totals into ft
        auto densities = [&](int b, int pl, float (&ft)[Q], float& rr, float& rb, bool keep) {
            const bool pvalid = !p.wall_z || (pl >= 0 && pl < p.nz);
            if (!pvalid) return;
            const int plw = wrap_near(pl, p.nz);
            if (owned) {
                pull(b, plw, slot(pl), otx, oty, ft, rr, rb, keep);
                phi_at(slot(pl), otx, oty) = colour(rr, rb);
            }
            if (ring) {
                float dummy[Q], a, c;
                pull(b, plw, slot(pl), rtx, rty, dummy, a, c, false);
                phi_at(slot(pl), rtx, rty) = colour(a, c);
            }
        };

        // ---- ring of source-node data of plane pl: element e of the (TX+4) x (TY+4)
        // box of source columns, wrapped on periodic axes, clamped at walls (values
        // beyond a wall are never read: those links bounce back). Each thread holds
        // elements tid and tid + NT; their in-plane offsets are worked out once per
        // segment: into the unpadded colour field (deviation storage) or into a padded
        // population block (the reduced form's coefficients), -1 for none.
        int ring_xy[2] = {-1, -1};
        if constexpr (RING) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int e = tid + j * NT;
                if (e >= LN) break;
                const int r = e / G::LW, c = e - r * G::LW;
                const int gx = wrap_near(x0 - 2 + c, p.nx);
                int gy = y0 - 2 + r;
                gy = p.wall_y ? min(max(gy, 0), p.ny - 1) : wrap_near(gy, p.ny);
                ring_xy[j] = G::RED ? (gy + 2) * p.pitch + gx + PADX : gy * p.nx + gx;
            }
        }
        auto ring_z = [&](int pl) {
            return p.wall_z ? min(max(pl, 0), p.nz - 1) : wrap_near(pl, p.nz);
        };
        // lagged colour field (deviation storage)
        auto lag_load = [&](int pl, int j) -> float {
            if (ring_xy[j] < 0) return 0.0f;
            return __ldg(p.phi_lag + (size_t)ring_z(pl) * plane + ring_xy[j]);
        };
        float lag_reg0 = 0.f, lag_reg1 = 0.f;   // plane fetched ahead of its slot store
        // reduced form: the coefficients of the same source columns of plane pl (the
        // step's input, read in place)
        float aux_reg[2][Q5_AUX];
        auto aux_fetch = [&](int pl) {
            if constexpr (G::RED) {
                const size_t base = (size_t)ring_z(pl) * p.plane_p;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (ring_xy[j] < 0) break;
#pragma unroll
                    for (int k = 0; k < Q5_AUX; ++k)
                        aux_reg[j][k] = St::coef(fin, p.P, base + ring_xy[j], k);
                }
            }
        };
        auto lag_fetch = [&](int pl) {
            if constexpr (G::RED) {
                aux_fetch(pl);
            } else {
                lag_reg0 = lag_load(pl, 0);
                lag_reg1 = lag_load(pl, 1);
            }
        };
        auto lag_commit = [&](int pl) {
            if constexpr (G::RED) {
                float* d = slag + (size_t)slot(pl) * (Q5_AUX * LN);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (ring_xy[j] < 0) break;
                    const int e = tid + j * NT;
                    reinterpret_cast<float2*>(d)[e] = make_float2(aux_reg[j][0], aux_reg[j][1]);
#pragma unroll
                    for (int k = 2; k < Q5_AUX; ++k) d[k * LN + e] = aux_reg[j][k];
                }
            } else {
                float* d = slag + (size_t)slot(pl) * LN;
                d[tid] = lag_reg0;
                if (tid + NT < LN) d[tid + NT] = lag_reg1;
            }
        };

        const int gxn = x0 + otx, gyn = y0 + oty;
        const bool use_nc = p.A_nc > 0.0f;
        const size_t col = (size_t)gyn * p.nx + gxn;   // owned column (unpadded fields)
        const float fx_y = owned ? __ldg(p.fx_row + gyn) : 0.0f;
        const bool ylo = p.wall_y && gyn == 0, yhi = p.wall_y && gyn == p.ny - 1;

        if constexpr (SC) {
            // ---- Shan-Chen model. The ring holds the species densities of planes
            // z-1, z (and z+1 once pulled); the cohesive force of plane z needs those
            // of its 18 neighbours. Away from unit rate each species' populations are
            // needed by the collision; they are kept only for the plane being collided:
            // at the start of plane z the staged buffer holds plane z; its owned
            // populations are pulled, the buffer is refilled with plane z+1, whose
            // densities (tile + ring) complete the ring, and plane z is collided. (Plane
            // z+1 is pulled once more, whole, in its own turn.)
            auto rho_at = [&](int k, int sl, int tx, int ty) -> float& {
                return sphi[((k * 4 + sl) * SH + ty + 1) * SWP + tx + 1];
            };
            auto sc_densities = [&](int b, int pl) {
                const bool pvalid = !p.wall_z || (pl >= 0 && pl < p.nz);
                if (!pvalid) return;
                const int plw = wrap_near(pl, p.nz);
                float vr[Q], vb[Q], a, c;
                if (owned) {
                    pull_species(b, plw, slot(pl), otx, oty, vr, vb, a, c, false);
                    rho_at(0, slot(pl), otx, oty) = a;
                    rho_at(1, slot(pl), otx, oty) = c;
                }
                if (ring) {
                    pull_species(b, plw, slot(pl), rtx, rty, vr, vb, a, c, false);
                    rho_at(0, slot(pl), rtx, rty) = a;
                    rho_at(1, slot(pl), rtx, rty) = c;
                }
            };
            // cohesive velocity shifts F^k / rho_k = -G sum_i w_i rho_kbar(x + c_i) c_i of
            // the owned node of plane z (densities rr, rb) from the ring of planes
            // z-1 .. z+1: 3 sum_i w_i rho_k(x + c_i) c_i per species, a neighbour beyond
            // a wall taking the node's own density
            const float g3 = -p.G_sc * (1.0f / 3.0f);
            auto sc_shifts = [&](int z, float rr, float rb, float (&sr)[3], float (&sb)[3]) {
                const bool zlo = p.wall_z && z == 0, zhi = p.wall_z && z == p.nz - 1;
                const int s0 = slot(z - 1), s1 = slot(z), s2 = slot(z + 1);
                float ar[3] = {0.f, 0.f, 0.f}, ab[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (i == 9) continue;
                    const bool wall = (cy(i) < 0 && ylo) || (cy(i) > 0 && yhi) ||
                                      (cz(i) < 0 && zlo) || (cz(i) > 0 && zhi);
                    const int sl = cz(i) < 0 ? s0 : (cz(i) > 0 ? s2 : s1);
                    const float nr = wall ? rr : rho_at(0, sl, otx + cx(i), oty + cy(i));
                    const float nb = wall ? rb : rho_at(1, sl, otx + cx(i), oty + cy(i));
                    grad_add(i, nr, ar[0], ar[1], ar[2]);
                    grad_add(i, nb, ab[0], ab[1], ab[2]);
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sr[a] = g3 * ab[a];
                    sb[a] = g3 * ar[a];
                }
            };
            if constexpr (UnitOmega) {
                // ---- unit rate (omega = 1): the collision needs only each node's
                // densities and momentum, not its populations, so the march takes the
                // colour-gradient form: each turn pulls plane z+1 once (tile and ring
                // densities into the ring, the owned node's densities and momentum into
                // registers) while the copy of plane z+2 is in flight, then collides z.
                auto sc_pull = [&](int b, int pl, float& rr, float& rb, float (&j)[3]) {
                    const bool pvalid = !p.wall_z || (pl >= 0 && pl < p.nz);
                    if (!pvalid) return;
                    const int plw = wrap_near(pl, p.nz);
                    float vr[Q], vb[Q], a, c;
                    if (owned) {
                        pull_species(b, plw, slot(pl), otx, oty, vr, vb, rr, rb, true);
                        sc_momentum(vr, vb, j[0], j[1], j[2]);
                        rho_at(0, slot(pl), otx, oty) = rr;
                        rho_at(1, slot(pl), otx, oty) = rb;
                    }
                    if (ring) {
                        pull_species(b, plw, slot(pl), rtx, rty, vr, vb, a, c, false);
                        rho_at(0, slot(pl), rtx, rty) = a;
                        rho_at(1, slot(pl), rtx, rty) = c;
                    }
                };
                float c_rr = 0.f, c_rb = 0.f, c_j[3] = {0.f, 0.f, 0.f};
                float n_rr = 0.f, n_rb = 0.f, n_j[3] = {0.f, 0.f, 0.f};
                // lag planes zb-2 .. zb (deviation storage), then each turn z stores lag
                // plane z+3 into the slot of z-1, as in the colour-gradient march
                if (G::DEV) {
                    for (int q = -2; q <= 0; ++q) {
                        lag_fetch(zb + q);
                        lag_commit(zb + q);
                    }
                    __syncthreads();
                }
                fence_proxy_async();
                issue(0, zb - 1);
                const float none[Q] = {};   // populations: unused at unit rate
                for (int z = zb - 2; z < ze; ++z) {
                    if (G::DEV) lag_fetch(z + 3);
                    wait(0);
                    sc_pull(0, z + 1, n_rr, n_rb, n_j);
                    if (G::DEV) lag_commit(z + 3);
                    if (my_st >= 0) bulk_wait_read();   // the output tile of plane z-1 has been read
                    __syncthreads();
                    fence_proxy_async();
                    if (z + 2 <= ze) issue(0, z + 2);
                    if (z >= zb) {
                        if (owned && !failed) {
                            float sr[3], sb[3];
                            sc_shifts(z, c_rr, c_rb, sr, sb);
                            const float phic = colour(c_rr, c_rb);
                            const SmemEmit<St, TX * TY> em{sout + oty * TX + otx};
                            sc_collide_moments<St, true>(p, none, none, c_rr, c_rb, c_j[0], c_j[1],
                                                         c_j[2], phic, sr, sb, fx_y, p.gy, p.gz, em);
                            p.phi_out[(size_t)z * plane + col] = phic;
                        }
                        fence_proxy_async();
                        __syncthreads();
                        if (my_st >= 0) {
                            tma_store_4d(fout_map, x0 + PADX, y0 + 2, z, my_st,
                                         sout + (size_t)my_st * (TX * TY));
                            bulk_commit();
                        }
                    }
                    c_rr = n_rr;
                    c_rb = n_rb;
#pragma unroll
                    for (int a = 0; a < 3; ++a) c_j[a] = n_j[a];
                }
                continue;
            }
            // the march starts at plane zb-2: its first two turns only fill the ring with
            // the densities of zb-1 and zb (one copy of the pull code for the segment);
            // lag planes zb-2, zb-1 first, then each turn z stores lag plane z+2
            if (G::DEV) {
                for (int q = -2; q <= -1; ++q) {
                    lag_fetch(zb + q);
                    lag_commit(zb + q);
                }
                lag_fetch(zb);
                __syncthreads();
            }
            for (int z = zb - 2; z < ze; ++z) {
                // lag plane z+2 goes to the slot of z-2, last read in the previous plane
                if (G::DEV) lag_commit(z + 2);
                float vr[Q], vb[Q], rr = 0.f, rb = 0.f;
                if (z >= zb && owned && !failed)
                    pull_species(0, z, slot(z), otx, oty, vr, vb, rr, rb, true);
                if (my_st >= 0) bulk_wait_read();   // the output tile of plane z-1 has been read
                __syncthreads();                  // staged plane z consumed
                fence_proxy_async();
                issue(0, z + 1);
                if (G::DEV) lag_fetch(z + 3);
                wait(0);
                sc_densities(0, z + 1);
                __syncthreads();                  // densities of plane z+1 in the ring
                if (z < zb) continue;
                if (owned && !failed) {
                    float sr[3], sb[3];
                    sc_shifts(z, rr, rb, sr, sb);
                    const float phic = colour(rr, rb);
                    const SmemEmit<St, TX * TY> em{sout + oty * TX + otx};
                    sc_collide_store<St, UnitOmega>(p, vr, vb, rr, rb, phic, sr, sb, fx_y, p.gy,
                                                    p.gz, em);
                    p.phi_out[(size_t)z * plane + col] = phic;
                }
                fence_proxy_async();
                __syncthreads();
                if (my_st >= 0) {
                    tma_store_4d(fout_map, x0 + PADX, y0 + 2, z, my_st, sout + (size_t)my_st * (TX * TY));
                    bulk_commit();
                }
            }
            continue;
        }

        // one plane of the march: densities of plane z+1 into (nx_f, nx_rr, nx_rb), then
        // the collision of plane z from (cu, cu_rr, cu_rb); A_h is carried in ah_c
        // (planes zb-2 and zb-1 only fill the ring: the march starts there, so that one
        // copy of the pull code serves the whole segment)
        auto march = [&](int z, float (&cu)[Q], float cu_rr, float cu_rb, float (&nx_f)[Q],
                         float& nx_rr, float& nx_rb, float& ah_c) {
            // plane z+1 is in the staging buffer (issued after the previous barrier);
            // plane z+2 is issued right after this plane's barrier frees the buffer
            const int bn = 0;
            const float ah_nxt = (owned && use_nc && z + 1 >= zb && z + 1 < ze)
                                     ? p.ah[(size_t)(z + 1) * plane + col]
                                     : 0.0f;
            // lag plane z+3 goes to the slot of plane z-1, last read before the barrier
            // of the previous plane; the densities of z+1 read planes z .. z+2. It is
            // fetched here and stored after those densities, which hide the latency.
            if (RING) lag_fetch(z + 3);
            wait(bn);
            densities(bn, z + 1, nx_f, nx_rr, nx_rb, true);
            if constexpr (UnitOmega) {
                // unit rate: the collision needs only the momentum of the populations,
                // which is all that is carried to the next turn (in nx_f[0 .. 2])
                if (owned) {
                    float jx, jy, jz;
                    cg_momentum(nx_f, jx, jy, jz);
                    nx_f[0] = jx;
                    nx_f[1] = jy;
                    nx_f[2] = jz;
                }
            }
            if (RING) lag_commit(z + 3);
            if (my_st >= 0) bulk_wait_read();   // the output tile of plane z-1 has been read
            __syncthreads();
            fence_proxy_async();
            if (z + 2 <= ze) issue(0, z + 2);
            if (z < zb) {
                ah_c = ah_nxt;
                return;
            }
            if (owned && !failed) {
                const bool zlo = p.wall_z && z == 0, zhi = p.wall_z && z == p.nz - 1;
                const int s0 = slot(z - 1), s1 = slot(z), s2 = slot(z + 1);
                const float phic = phi_at(s1, otx, oty);
                // isotropic colour gradient, 3 w_i = 1/6 (faces), 1/12 (edges); a
                // neighbour beyond a wall takes the centre value
                float Gx = 0.f, Gy = 0.f, Gz = 0.f;
                if (!(ylo || yhi || zlo || zhi)) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (i == 9) continue;
                        const int sl = cz(i) < 0 ? s0 : (cz(i) > 0 ? s2 : s1);
                        grad_add(i, phi_at(sl, otx + cx(i), oty + cy(i)), Gx, Gy, Gz);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (i == 9) continue;
                        const bool wall = (cy(i) < 0 && ylo) || (cy(i) > 0 && yhi) ||
                                          (cz(i) < 0 && zlo) || (cz(i) > 0 && zhi);
                        const int sl = cz(i) < 0 ? s0 : (cz(i) > 0 ? s2 : s1);
                        grad_add(i, wall ? phic : phi_at(sl, otx + cx(i), oty + cy(i)), Gx, Gy, Gz);
                    }
                }
                const size_t node = (size_t)z * plane + col;
                float Fx = fx_y, Fy = p.gy, Fz = p.gz;
                if (use_nc) {
                    // near-contact force A_h G, A_h measured by the near-contact pass
                    // (which writes every node's A_h)
                    if (ah_c != 0.0f) {
                        Fx += ah_c * Gx;
                        Fy += ah_c * Gy;
                        Fz += ah_c * Gz;
                    }
                }
                // outputs go to the shared output tile; the tile is stored below
                const SmemEmit<St, TX * TY> em{sout + oty * TX + otx};
                if constexpr (UnitOmega)
                    collide_moments<St, true>(p, cu, cu_rr, cu_rb, cu[0], cu[1], cu[2], phic, Gx,
                                              Gy, Gz, Fx, Fy, Fz, em);
                else
                    collide_store<St, UnitOmega>(p, cu, cu_rr, cu_rb, phic, Gx, Gy, Gz, Fx, Fy, Fz, em);
                p.phi_out[node] = phic;
            }
            // store the output tile of plane z: 2Q tensor copies of TX x TY, clipped by
            // the store map at the lattice edge (to 16 bytes: ghost copies are written
            // afterwards by the fill pass); the tile is rewritten only after these
            // copies have read it
            fence_proxy_async();
            __syncthreads();
            if (my_st >= 0) {
                tma_store_4d(fout_map, x0 + PADX, y0 + 2, z, my_st, sout + (size_t)my_st * (TX * TY));
                bulk_commit();
            }
            ah_c = ah_nxt;
        };

        float fa[Q], fb[Q];
        float a_rr = 0.f, a_rb = 0.f, b_rr = 0.f, b_rb = 0.f;
        float ah_c = 0.0f;   // A_h of the plane being collided, loaded one plane ahead

        // ---- lag (or coefficient) planes zb-2 .. zb for the densities of zb-1 (each
        // plane z of the march then stores plane z+3 into the slot of z-1), and the
        // copy of plane zb-1
        if (RING) {
            for (int q = -2; q <= 0; ++q) {
                lag_fetch(zb + q);
                lag_commit(zb + q);
            }
            __syncthreads();
        }
        fence_proxy_async();
        issue(0, zb - 1);

        // ---- the march: plane z is collided from fa while plane z+1 is pulled into fb
        // (at unit rate only fa[0 .. 2], the momentum, is carried)
        for (int z = zb - 2; z < ze; ++z) {
            march(z, fa, a_rr, a_rb, fb, b_rr, b_rb, ah_c);
#pragma unroll
            for (int i = 0; i < (UnitOmega ? 3 : Q); ++i) fa[i] = fb[i];
            a_rr = b_rr;
            a_rb = b_rb;
        }
    }
    grid_dep_launch();
    if (my_st >= 0) bulk_wait_all();   // output tiles written before the CTA exits
    if (failed) {
        // give copies still in flight into this CTA's shared memory a bounded chance
        // to land before the CTA exits
        for (int b = 0; b < STAGES; ++b)
            for (uint32_t it = 0; it < (1u << 20); ++it)
                if (mbar_try_wait(&bars[b], (parity >> b) & 1u)) break;
    }
}

template <class St, bool UnitOmega, bool SC>
__global__ void __launch_bounds__(NT, CTAS_PER_SM)
step_kernel(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap fin_map,
            const __grid_constant__ CUtensorMap fout_map) {
    step_body<St, UnitOmega, SC>(p, &fin_map, &fout_map, (int)blockIdx.x);
}

// Several lattices in one launch: CTA b belongs to the last lattice whose first CTA
// is <= b. Its parameters are copied to shared memory once; its tensor maps are read
// from the table (global memory).
template <class St, bool UnitOmega, bool SC>
__global__ void __launch_bounds__(NT, CTAS_PER_SM)
step_kernel_batched(const BatchLattice* __restrict__ tab, int nlat) {
    __shared__ StepParams sp;
    __shared__ int lat;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].cta_begin <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        lat = lo;
    }
    __syncthreads();
    const BatchLattice& L = tab[lat];
    {
        const int* src = reinterpret_cast<const int*>(&L.p);
        int* dst = reinterpret_cast<int*>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(StepParams) / sizeof(int)); i += blockDim.x)
            dst[i] = src[i];
    }
    __syncthreads();
    step_body<St, UnitOmega, SC>(sp, &L.in_map, &L.out_map, (int)blockIdx.x - L.cta_begin);
}

// ---------------------------------------------------------------- in-place (AA) step
// With in-place storage (one population copy, see aa_slot) a step is two passes over
// the nodes:
//  aa_phi_kernel: each node's post-stream species densities from the slots its
//    populations are in, and its colour field into phi_out (reads only);
//  aa_collide_kernel: the same densities again, the isotropic gradient of phi_out,
//    the forces, and the collision of the fused kernel (the same source in the same
//    order), its outputs written to the node's own slots in the other layout.
// Work items are row segments of AA_W nodes (x0 .. x0 + AA_W - 1 of row (y, z)), one
// per CTA at a time, one node per thread: everything that depends on the row (the
// source and target rows of every direction, wall tests) is the same for the whole
// CTA, and a thread adds only its wrapped x offset. Both layouts run the same kernels
// (the layout is an argument), so a state reached in either layout steps on with the
// same arithmetic. Colour-gradient model, full storage forms (FP32, FP16/BF16 deviations),
// walls at rest. Bytes per node and step: the populations read twice and written
// once (1.5x the two-copy step's) for half its memory.
constexpr int AA_W = 128;

// Node (x, y, z) of a row segment, with the row's index bases.
struct AaNode {
    int x, y, z;
    unsigned self;   // padded index (population blocks; < 2^31, checked at creation)
    unsigned pself;  // unpadded index (colour fields, A_h)
};
// Index offsets of node n + (dx, dy, dz) (|d| <= 1) from n: padded (off) and
// unpadded (poff), wrapped on periodic axes; false if it lies beyond a wall. The y and
// z parts depend on the row only (the same for the whole CTA); x adds the lane's part.
__device__ __forceinline__ bool aa_offset(const StepParams& p, const AaNode& n, int dx, int dy,
                                          int dz, int& off, int& poff) {
    const int planeP = p.nyp * p.pitch, plane = p.ny * p.nx;
    off = 0;
    poff = 0;
    if (dz != 0) {
        const int v = n.z + dz;
        int w = dz;
        if (v < 0 || v >= p.nz) {
            if (p.wall_z) return false;
            w = v < 0 ? p.nz - 1 : 1 - p.nz;
        }
        off += w * planeP;
        poff += w * plane;
    }
    if (dy != 0) {
        const int v = n.y + dy;
        int w = dy;
        if (v < 0 || v >= p.ny) {
            if (p.wall_y) return false;
            w = v < 0 ? p.ny - 1 : 1 - p.ny;
        }
        off += w * p.pitch;
        poff += w * p.nx;
    }
    if (dx != 0) {
        const int v = n.x + dx;
        const int w = v < 0 ? p.nx - 1 : (v >= p.nx ? 1 - p.nx : dx);
        off += w;
        poff += w;
    }
    return true;
}

// Post-stream populations f_i(x) = f*_i(x - c_i) of node n (from beyond a wall
// f*_opp(i)(x)) from the state in layout L, and the species densities. Deviation
// storage decodes each value against the lagged colour field of the node that wrote
// it. Every value is loaded before any is decoded (all loads in flight at once).
template <class St>
__device__ __forceinline__ void aa_pull(const StepParams& p, int L, const AaNode& n,
                                        float (&vr)[Q], float (&vb)[Q], float& rr, float& rb) {
    using T = typename St::T;
    const T* f = static_cast<const T*>(p.fin);
    T raw_r[Q], raw_b[Q];
    float ph[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // the writer: n - c_i, or n itself for a link from beyond a wall
        int off, poff;
        const bool in = aa_offset(p, n, -cx(i), -cy(i), -cz(i), off, poff);
        unsigned idx = n.self;
        const T *fr = f + (size_t)i * p.P, *fb = f + (size_t)(Q + i) * p.P;
        if (L == 0 && in) {           // f*_i of the writer, in its slot (opp(i), writer)
            idx = n.self + off;
            fr = f + (size_t)opp(i) * p.P;
            fb = f + (size_t)(Q + opp(i)) * p.P;
        }                             // else: the node's own slot (i, x)
        raw_r[i] = fr[idx];
        raw_b[i] = fb[idx];
        if (St::DEV) ph[i] = __ldg(p.phi_lag + (n.pself + (in ? poff : 0)));
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float rf_r = 0.f, rf_b = 0.f;
        if (St::DEV) {
            const float hw = wgt(i) * p.ref_half;
            rf_r = dev_ref(hw, ph[i], 0);
            rf_b = dev_ref(hw, ph[i], 1);
        }
        vr[i] = St::cvt(raw_r[i], rf_r);
        vb[i] = St::cvt(raw_b[i], rf_b);
    }
    rr = sum19(vr);
    rb = sum19(vb);
}

// Row segment t of the lattice: first node x0 of row (y, z), for t in [0, rows x
// segments per row).
__device__ __forceinline__ void aa_item(const StepParams& p, long long t, int& x0, int& y, int& z) {
    const int segs = (p.nx + AA_W - 1) / AA_W;
    const long long r = t / segs;
    x0 = (int)(t - r * segs) * AA_W;
    z = (int)(r / p.ny);
    y = (int)(r - (long long)z * p.ny);
}
__host__ __device__ inline long long aa_items(const StepParams& p) {
    return (long long)p.nz * p.ny * ((p.nx + AA_W - 1) / AA_W);
}

__device__ __forceinline__ AaNode aa_node(const StepParams& p, int x, int y, int z) {
    return AaNode{x, y, z, (unsigned)pidx(p.pitch, p.nyp, p.padx, x, y, z),
                  (unsigned)(((size_t)z * p.ny + y) * p.nx + x)};
}

template <class St>
__global__ void __launch_bounds__(AA_W) aa_phi_kernel(const StepParams p, int L) {
    grid_dep_wait();
    const long long items = aa_items(p);
    for (long long t = blockIdx.x; t < items; t += gridDim.x) {
        int x0, y, z;
        aa_item(p, t, x0, y, z);
        const int x = x0 + (int)threadIdx.x;
        if (x >= p.nx) continue;
        const AaNode n = aa_node(p, x, y, z);
        float vr[Q], vb[Q], rr, rb;
        aa_pull<St>(p, L, n, vr, vb, rr, rb);
        p.phi_out[n.pself] = colour(rr, rb);
    }
    grid_dep_launch();
}

// Emitter of the collision for in-place storage: output block k (species k / Q,
// direction k % Q) to the node's slot of that direction in layout LO.
template <class St>
struct AaEmit {
    typename St::T* f;
    const StepParams* p;
    AaNode n;
    int LO;
    __device__ __forceinline__ void operator()(int k, float v, float ref) const {
        const int sp = k >= Q ? 1 : 0, i = k - sp * Q;
        unsigned idx = n.self;
        typename St::T* fd = f + (size_t)(sp * Q + opp(i)) * p->P;
        int off, poff;
        if (LO == 1 && aa_offset(*p, n, cx(i), cy(i), cz(i), off, poff)) {
            idx = n.self + off;       // (i, x + c_i) unless that lies beyond a wall
            fd = f + (size_t)(sp * Q + i) * p->P;
        }
        fd[idx] = St::enc(v, ref);
    }
    __device__ __forceinline__ void coef(int, float) const {}
};

// Isotropic colour gradient of phi at node n (a neighbour beyond a wall takes the
// centre value): the terms of gradient_global in the same order.
__device__ __forceinline__ void aa_gradient(const StepParams& p, const float* phi, const AaNode& n,
                                            float& Gx, float& Gy, float& Gz) {
    float v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int off, poff;
        v[i] = __ldg(phi + (n.pself + (aa_offset(p, n, cx(i), cy(i), cz(i), off, poff) ? poff : 0)));
    }
    Gx = Gy = Gz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (i != 9) grad_add(i, v[i], Gx, Gy, Gz);
}

template <class St, bool UnitOmega>
__global__ void __launch_bounds__(AA_W) aa_collide_kernel(const StepParams p, int L) {
    grid_dep_wait();
    const long long items = aa_items(p);
    const bool use_nc = p.A_nc > 0.0f;
    for (long long t = blockIdx.x; t < items; t += gridDim.x) {
        int x0, y, z;
        aa_item(p, t, x0, y, z);
        const int x = x0 + (int)threadIdx.x;
        if (x >= p.nx) continue;
        const AaNode n = aa_node(p, x, y, z);
        float vr[Q], vb[Q], rr, rb;
        aa_pull<St>(p, L, n, vr, vb, rr, rb);
        float ft[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) ft[i] = vr[i] + vb[i];
        const float phic = colour(rr, rb);
        float Gx, Gy, Gz;
        aa_gradient(p, p.phi_out, n, Gx, Gy, Gz);
        float Fx = __ldg(p.fx_row + y), Fy = p.gy, Fz = p.gz;
        if (use_nc) {
            const float ah = __ldg(p.ah + n.pself);
            if (ah != 0.0f) {
                Fx += ah * Gx;
                Fy += ah * Gy;
                Fz += ah * Gz;
            }
        }
        const AaEmit<St> em{static_cast<typename St::T*>(p.fout), &p, n, L ^ 1};
        if constexpr (UnitOmega) {
            float jx, jy, jz;
            cg_momentum(ft, jx, jy, jz);
            collide_moments<St, true>(p, ft, rr, rb, jx, jy, jz, phic, Gx, Gy, Gz, Fx, Fy, Fz, em);
        } else {
            collide_store<St, false>(p, ft, rr, rb, phic, Gx, Gy, Gz, Fx, Fy, Fz, em);
        }
    }
    grid_dep_launch();
}

// ---------------------------------------------------------------- ghost fill
// Ghost copies of the periodic axes, in warp tasks (each task's indices are worked
// out once; the lanes sweep a row or a column of rows):
//  part 1, one task per (block k, plane z), lanes over the rows y: x ghosts -2, -1 <-
//          nodes nx-2, nx-1 and nx, nx+1 <- nodes 0, 1, each side as one aligned pair
//          of elements when nx is even (two elements otherwise);
//  part 2 (periodic y only), one task per (k, z, ghost row -2, -1, ny, ny+1), lanes
//          over x = -2 .. nx+1: each element from the wrapped node (corners included).
// With K = p.ghost_arrays streamed blocks (2Q, or Q in the reduced form: its
// coefficient blocks are read in place), part 1 has K nz tasks, part 2 K nz 4.
// (Writing the whole 32-byte ghost sectors instead of the pairs measured no faster:
// the fill waits on its loads.)
__host__ __device__ inline long long ghost_part1(const StepParams& p) {
    return (long long)p.ghost_arrays * p.nz;
}
__host__ __device__ inline long long ghost_work(const StepParams& p) {
    return ghost_part1(p) + (p.wall_y ? 0 : (long long)p.ghost_arrays * p.nz * 4);
}

template <int B> struct PairOf;
template <> struct PairOf<2> { using type = unsigned int; };
template <> struct PairOf<4> { using type = unsigned long long; };

template <class St>
__device__ __forceinline__ void ghost_task(typename St::T* f, const StepParams& p, long long t,
                                           int lane) {
    using T = typename St::T;
    using Pair = typename PairOf<sizeof(T)>::type;
    const long long n1 = ghost_part1(p);
    if (t < n1) {
        const int k = (int)(t / p.nz), z = (int)(t - (long long)k * p.nz);
        T* blk = f + (size_t)k * p.P;
        if ((p.nx & 1) == 0 && p.nx >= 2) {
            // row[-2], row[-1] <- row[nx-2], row[nx-1]; row[nx], row[nx+1] <- row[0], row[1]
            // (GB rows at a time: every load of a batch is issued before its stores)
            constexpr int GB = 4;
            for (int y0 = lane; y0 < p.ny; y0 += 32 * GB) {
                Pair a[GB], b[GB];
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    const int y = y0 + 32 * g;
                    if (y < p.ny) {
                        const T* row = blk + pidx(p.pitch, p.nyp, p.padx, 0, y, z);
                        a[g] = *reinterpret_cast<const Pair*>(row + p.nx - 2);
                        b[g] = *reinterpret_cast<const Pair*>(row);
                    }
                }
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    const int y = y0 + 32 * g;
                    if (y < p.ny) {
                        T* row = blk + pidx(p.pitch, p.nyp, p.padx, 0, y, z);
                        *reinterpret_cast<Pair*>(row - 2) = a[g];
                        *reinterpret_cast<Pair*>(row + p.nx) = b[g];
                    }
                }
            }
            return;
        }
        for (int y = lane; y < p.ny; y += 32) {   // odd nx: element by element
            T* row = blk + pidx(p.pitch, p.nyp, p.padx, 0, y, z);   // node x = 0
            const T a0 = row[wrap_near(-2, p.nx)], a1 = row[wrap_near(-1, p.nx)];
            const T b0 = row[wrap_near(p.nx, p.nx)], b1 = row[wrap_near(p.nx + 1, p.nx)];
            row[-2] = a0;
            row[-1] = a1;
            row[p.nx] = b0;
            row[p.nx + 1] = b1;
        }
        return;
    }
    const long long j = t - n1;
    const int r = (int)(j & 3);
    const long long kz = j >> 2;
    const int k = (int)(kz / p.nz), z = (int)(kz - (long long)k * p.nz);
    const int y = r < 2 ? r - 2 : p.ny + r - 2;
    T* blk = f + (size_t)k * p.P;
    T* dst = blk + pidx(p.pitch, p.nyp, p.padx, 0, y, z);
    const T* src = blk + pidx(p.pitch, p.nyp, p.padx, 0, wrap_near(y, p.ny), z);
    constexpr int GB = 4;
    for (int x0 = lane - 2; x0 < p.nx + 2; x0 += 32 * GB) {
        T v[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int x = x0 + 32 * g;
            if (x < p.nx + 2) v[g] = src[wrap_near(x, p.nx)];
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int x = x0 + 32 * g;
            if (x < p.nx + 2) dst[x] = v[g];
        }
    }
}

template <class St>
__global__ void ghost_fill_kernel(typename St::T* f, const StepParams p) {
    grid_dep_wait();
    const long long total = ghost_work(p);
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < total;
         t += nw)
        ghost_task<St>(f, p, t, lane);
    grid_dep_launch();
}

// Ghost copies of every lattice of a batch: task t belongs to the last lattice whose
// first task is <= t.
template <class St>
__global__ void ghost_fill_batched(const BatchLattice* __restrict__ tab, int nlat,
                                   long long total) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < total;
         t += nw) {
        int lo = 0, hi = nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].ghost_begin <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchLattice& L = tab[lo];
        ghost_task<St>(static_cast<typename St::T*>(L.fout), L.p, t - L.ghost_begin, lane);
    }
}

// ---------------------------------------------------------------- near-contact pass, block form
// A_h of every node from the lagged colour field, one NB_X x NB_Y x NB_Z block of nodes
// at a time. A work item is a column of blocks (bx, by) and a segment of up to nc_seg
// consecutive blocks along z (persistent CTAs, items in x-fastest order, so that the
// CTAs resident at one time work on neighbouring columns and their halos come from L2).
// The block's lagged field and a halo of H nodes around it -- the farthest trilinear
// corner a ray of samples up to t = h_cut + 2 reaches is floor(h_cut) + 3 <= H nodes
// away -- sit in a shared-memory cube, kept as a ring of SZ planes along z: the first
// block of a segment copies all of its planes, every later block only the NB_Z planes
// that enter its window (a third of the copying). Each plane is one TMA tensor copy
// where the cube lies inside the lattice in x and y (a walled y axis may reach past its
// walls: zero fill, never read), else asynchronous copies wrapped on periodic axes and
// clamped at walls. Two CTAs share an SM, one cube each (the halo-9 cube and the ray
// list take 112 KB): while one waits for its copy or at a barrier between the phases
// below, the other works. Then:
//  1. every node's lagged gradient G' is evaluated in the cube, with the same
//     expression in the same order as the step kernel's gradient (so the same bits); a
//     node with |G'| >= 1e-3 is listed, every other node's A_h is final (0);
//  2. the listed rays, one per thread: every sample is interpolated from the cube (the
//     same cells, weights and interpolation order as the oracle's definition, in FP32)
//     and classified by sign, all samples of every ray in turn, so that the lanes of a
//     warp stay together; A_h follows from the sign masks and the four samples around
//     the two crossings (NcRay::measure).
// Every node's A_h is written (0 where no film is within h_cut): the field needs no
// clearing between passes and no candidate list. The kernel also writes the ghost
// copies of the step's input populations (two-copy storage): a warp with no ray left
// in a block's last round takes one ghost task, and the CTA's remaining tasks follow
// its last block.
constexpr int NB_X = 16, NB_Y = 8, NB_Z = 8, NB_NODES = NB_X * NB_Y * NB_Z;
constexpr int NB_THREADS = 512, NB_PER_THREAD = NB_NODES / NB_THREADS;

template <int H>
struct NcBlockGeo {
    static constexpr int HX = (H + 3) / 4 * 4;     // x halo, a multiple of 16 bytes
    static constexpr int SX = NB_X + 2 * HX, SY = NB_Y + 2 * H, SZ = NB_Z + 2 * H;
    static constexpr int ROWS = SY * SZ;
    static constexpr int CHUNKS = SX / 4;          // 16-byte chunks per cube row
    // floats per cube plane (SY rows of SX), padded so that every plane starts on a
    // 128-byte boundary (the destination of a tensor copy)
    static constexpr int PLANE = (SX * SY + 31) / 32 * 32;
    static constexpr size_t CUBE_BYTES = (size_t)PLANE * SZ * sizeof(float);
    // the mbarrier (4 slots), the list of the block's rays and its length
    static constexpr size_t FIXED = 4 * sizeof(unsigned long long) + (NB_NODES + 4) * sizeof(int);
    static constexpr size_t SMEM = CUBE_BYTES + FIXED;
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Row of the halo cube along a periodic (wrapped) or walled (clamped) axis.
__device__ __forceinline__ int halo_index(int a, int n, bool walled) {
    return walled ? min(max(a, 0), n - 1) : wrap_near(a, n);
}

// Ring slot of window plane k (0 <= k < 2 SZ) of a block whose window starts in slot
// zbase: the cube keeps the SZ planes of a block's window in a ring along z, so that
// the next block of the same column reuses the SZ - NB_Z planes they share.
template <int H>
__device__ __forceinline__ int ring_slot(int zbase, int k) {
    const int r = zbase + k;
    return r >= NcBlockGeo<H>::SZ ? r - NcBlockGeo<H>::SZ : r;
}

// Cell of a ray sample in the cube: ray_cell's corners and fractions, with the corner
// (ix0, iy0, iz0) as offsets into the cube's ring: o0 in the plane of iz0, o1 in the
// plane of iz0 + 1 (the cube's copies of wrapped nodes make the other corners 1, SX
// and SX + 1 further on).
struct CubeCell {
    int o0, o1;
    float fx, fy, fz;
};
template <int H, bool W>
__device__ __forceinline__ void cube_cell(const StepParams& p, int y, int z, int y0, int z0,
                                          int lx, int ly, int lz, int zbase, float ox, float oy,
                                          float oz, CubeCell& c) {
    using G = NcBlockGeo<H>;
    const float flx = floorf(ox), fly = floorf(oy), flz = floorf(oz);
    c.fx = ox - flx;
    c.fy = oy - fly;
    c.fz = oz - flz;
    const int cx0 = lx + G::HX + (int)flx;
    int cy0 = ly + H + (int)fly, cz0 = lz + H + (int)flz;
    if (W && p.wall_y && y + (int)fly == p.ny - 1) {   // on the last node: the cell below, fy = 1
        cy0 = p.ny - 2 - y0 + H;
        c.fy = 1.0f;
    }
    if (W && p.wall_z && z + (int)flz == p.nz - 1) {
        cz0 = p.nz - 2 - z0 + H;
        c.fz = 1.0f;
    }
    const int r = cy0 * G::SX + cx0;
    c.o0 = ring_slot<H>(zbase, cz0) * G::PLANE + r;
    c.o1 = ring_slot<H>(zbase, cz0 + 1) * G::PLANE + r;
}
template <int H>
__device__ __forceinline__ void cube_corners(const float* cube, const CubeCell& c, float (&v)[8]) {
    using G = NcBlockGeo<H>;
    const float* b0 = cube + c.o0;
    const float* b1 = cube + c.o1;
    v[0] = b0[0];
    v[1] = b0[1];
    v[2] = b0[G::SX];
    v[3] = b0[G::SX + 1];
    v[4] = b1[0];
    v[5] = b1[1];
    v[6] = b1[G::SX];
    v[7] = b1[G::SX + 1];
}
__device__ __forceinline__ float cube_interp(const CubeCell& c, const float (&v)[8]) {
    const float c0 = ray_lerp(ray_lerp(v[0], v[1], c.fx), ray_lerp(v[2], v[3], c.fx), c.fy);
    const float c1 = ray_lerp(ray_lerp(v[4], v[5], c.fx), ray_lerp(v[6], v[7], c.fx), c.fy);
    return ray_lerp(c0, c1, c.fz);
}

// Lagged gradient of block node (lx, ly, lz) = lattice node (x, y, z) from the cube: the
// terms of gradient_global in its order; a neighbour beyond a wall takes the centre value.
template <int H, bool W>
__device__ __forceinline__ void cube_gradient(const StepParams& p, const float* cube, int x, int y,
                                              int z, int lx, int ly, int lz, int zbase, float& Gx,
                                              float& Gy, float& Gz) {
    using G = NcBlockGeo<H>;
    const int r = (ly + H) * G::SX + (lx + G::HX);
    const float* pm = cube + ring_slot<H>(zbase, lz + H - 1) * G::PLANE + r;
    const float* p0 = cube + ring_slot<H>(zbase, lz + H) * G::PLANE + r;
    const float* pp = cube + ring_slot<H>(zbase, lz + H + 1) * G::PLANE + r;
    const float phic = p0[0];
    const bool ylo = W && p.wall_y && y == 0, yhi = W && p.wall_y && y == p.ny - 1;
    const bool zlo = W && p.wall_z && z == 0, zhi = W && p.wall_z && z == p.nz - 1;
    Gx = Gy = Gz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (i == 9) continue;
        const bool wall = (cy(i) < 0 && ylo) || (cy(i) > 0 && yhi) || (cz(i) < 0 && zlo) ||
                          (cz(i) > 0 && zhi);
        const float* pl = cz(i) < 0 ? pm : (cz(i) > 0 ? pp : p0);
        const float v = wall ? phic : pl[cy(i) * G::SX + cx(i)];
        grad_add(i, v, Gx, Gy, Gz);
    }
}

// Work item t of a lattice's near-contact pass: block column (bx, by) and the blocks
// bz0 .. bz1-1 of its segment along z.
__device__ __forceinline__ void nc_item(const StepParams& p, long long t, int& bx, int& by, int& bz0,
                                        int& bz1) {
    const int bxn = (p.nx + NB_X - 1) / NB_X, byn = (p.ny + NB_Y - 1) / NB_Y;
    const int bzn = (p.nz + NB_Z - 1) / NB_Z, seg = p.nc_seg > 0 ? p.nc_seg : 1;
    bx = (int)(t % bxn);
    const long long r = t / bxn;
    by = (int)(r % byn);
    bz0 = (int)(r / byn) * seg;
    bz1 = min(bzn, bz0 + seg);
}

// Starts the copy of window planes k0 .. SZ-1 of the block at (x0, y0, z0) into their
// ring slots: one tensor copy per plane by thread 0 (completing on `bar`, which thread
// 0 arrives at once per fill, with 0 bytes when it is not used) where the cube lies
// inside the lattice in x and y (a walled y axis may reach past its walls: zero fill,
// never read), else the asynchronous copies of every thread, wrapped on periodic axes
// and clamped at walls (one commit group per fill). Planes beyond a z wall are clamped
// (never read).
template <int H>
__device__ __forceinline__ void nc_fill_planes(const StepParams& p, const CUtensorMap* map,
                                               bool tma_ok, int x0, int y0, int z0, int k0,
                                               int zbase, float* cube, unsigned long long* bar) {
    using G = NcBlockGeo<H>;
    const bool inside = tma_ok && x0 >= G::HX && x0 + NB_X + G::HX <= p.nx &&
                        (p.wall_y || (y0 >= H && y0 + NB_Y + H <= p.ny));
    const int tid = threadIdx.x;
    if (inside) {
        if (tid == 0) {
            // (each copy delivers SY rows of SX values: a plane without its padding)
            mbar_arrive_tx(bar, (uint32_t)((G::SZ - k0) * G::SX * G::SY * sizeof(float)));
            for (int k = k0; k < G::SZ; ++k)
                tma_load_3d(cube + (size_t)ring_slot<H>(zbase, k) * G::PLANE, map, x0 - G::HX,
                            y0 - H, halo_index(z0 - H + k, p.nz, p.wall_z), bar);
        }
    } else {
        if (tid == 0) mbar_arrive_tx(bar, 0u);
        const int rows = (G::SZ - k0) * G::SY;
        if ((p.nx & 3) == 0) {   // 16-byte chunks then never straddle the periodic seam
            for (int e = tid; e < rows * G::CHUNKS; e += NB_THREADS) {
                const int c = e % G::CHUNKS, row = e / G::CHUNKS;
                const int ly = row % G::SY, k = k0 + row / G::SY;
                const int gy = halo_index(y0 - H + ly, p.ny, p.wall_y);
                const int gz = halo_index(z0 - H + k, p.nz, p.wall_z);
                const int gx = wrap_near(x0 - G::HX + 4 * c, p.nx);
                cp_async16(cube + (size_t)ring_slot<H>(zbase, k) * G::PLANE + ly * G::SX + 4 * c,
                           p.phi_lag + ((size_t)gz * p.ny + gy) * p.nx + gx);
            }
        } else {
            for (int e = tid; e < rows * G::SX; e += NB_THREADS) {
                const int c = e % G::SX, row = e / G::SX;
                const int ly = row % G::SY, k = k0 + row / G::SY;
                const int gy = halo_index(y0 - H + ly, p.ny, p.wall_y);
                const int gz = halo_index(z0 - H + k, p.nz, p.wall_z);
                const int gx = wrap_near(x0 - G::HX + c, p.nx);
                cp_async4(cube + (size_t)ring_slot<H>(zbase, k) * G::PLANE + ly * G::SX + c,
                          p.phi_lag + ((size_t)gz * p.ny + gy) * p.nx + gx);
            }
        }
    }
    cp_async_commit();
}

// One ray of the block pass: node, direction, and A_h from its samples.
struct NcRay {
    int lx, ly, lz, x, y, z, s_end, zb;
    float nx_, ny_, nz_, a;
    template <int H, bool W>
    __device__ __forceinline__ void start(const StepParams& p, const float* cube, int idx, int x0,
                                          int y0, int z0, int zbase) {
        zb = zbase;
        lx = idx % NB_X;
        ly = (idx / NB_X) % NB_Y;
        lz = idx / (NB_X * NB_Y);
        x = x0 + lx;
        y = y0 + ly;
        z = z0 + lz;
        float Gx, Gy, Gz;
        cube_gradient<H, W>(p, cube, x, y, z, lx, ly, lz, zb, Gx, Gy, Gz);
        nc_ray(Gx, Gy, Gz, nx_, ny_, nz_);
        s_end = nc_sample_end(p, y, z, ny_, nz_);
        a = 0.0f;
    }
    // The lagged colour field at the sample at t, interpolated from the cube.
    template <int H, bool W>
    __device__ __forceinline__ float value(const StepParams& p, const float* cube, int y0, int z0,
                                           float t) const {
        CubeCell cell;
        cube_cell<H, W>(p, y, z, y0, z0, lx, ly, lz, zb, t * nx_, t * ny_, t * nz_, cell);
        float v[8];
        cube_corners<H>(cube, cell, v);
        return cube_interp(cell, v);
    }
    // A_h of the film along the ray: the march of NcMarch over samples 0 .. s_end - 1,
    // evaluated from the samples' sign classes. Samples within kSignBand of zero carry
    // no sign and are skipped. The downward crossing is at the first negative sample j
    // whose previous signed sample jp is positive; the upward one at the first positive
    // sample k after j, whose previous signed sample kp is negative. The march stops
    // with A_h = 0 at a signed sample m between j and k with t_m - t_d >= h_cut, i.e.
    // when kp != j and t_kp - t_d >= h_cut; otherwise A_h = A_h(t_u - t_d), each
    // crossing located by linear interpolation between its two samples (the same
    // expressions as the march: the same bits).
    template <int H, bool W>
    __device__ __forceinline__ void measure(const StepParams& p, const float* cube, int y0, int z0) {
        uint32_t P = 0u, N = 0u;
        if (s_end == 19) {   // (h_cut = 6, no wall on the ray: every sample unrolled)
#pragma unroll
            for (int s = 0; s < 19; ++s) {
                const float v = value<H, W>(p, cube, y0, z0, -1.0f + 0.5f * (float)s);
                P |= (v > kSignBand ? 1u : 0u) << s;
                N |= (v < -kSignBand ? 1u : 0u) << s;
            }
        } else {
#pragma unroll 4
            for (int s = 0; s < s_end; ++s) {
                const float v = value<H, W>(p, cube, y0, z0, -1.0f + 0.5f * (float)s);
                P |= (v > kSignBand ? 1u : 0u) << s;
                N |= (v < -kSignBand ? 1u : 0u) << s;
            }
        }
        const uint32_t S = P | N;
        int jp = -1, j = -1;
        for (uint32_t m = S, prev = 32u; m != 0u; m &= m - 1u) {
            const uint32_t i = (uint32_t)(__ffs((int)m) - 1);
            if (prev < 32u && ((P >> prev) & 1u) && ((N >> i) & 1u)) {
                jp = (int)prev;
                j = (int)i;
                break;
            }
            prev = i;
        }
        if (j < 0) return;
        const uint32_t later = P & ~((2u << j) - 1u);   // positive samples after j
        if (later == 0u) return;
        const int k = __ffs((int)later) - 1;
        const int kp = 31 - __clz((int)(S & ((1u << k) - 1u)));
        const float t_jp = -1.0f + 0.5f * (float)jp, t_j = -1.0f + 0.5f * (float)j;
        const float v_jp = value<H, W>(p, cube, y0, z0, t_jp), v_j = value<H, W>(p, cube, y0, z0, t_j);
        const float t_d = t_jp + (t_j - t_jp) * v_jp / (v_jp - v_j);
        const float t_kp = -1.0f + 0.5f * (float)kp, t_k = -1.0f + 0.5f * (float)k;
        if (kp != j && t_kp - t_d >= p.h_cut) return;
        const float v_kp = value<H, W>(p, cube, y0, z0, t_kp), v_k = value<H, W>(p, cube, y0, z0, t_k);
        const float t_u = t_kp + (t_k - t_kp) * v_kp / (v_kp - v_k);
        a = A_h(p, t_u - t_d);
    }
    __device__ __forceinline__ void finish(const StepParams& p, size_t plane) {
        const size_t node = (size_t)z * plane + (size_t)y * p.nx + x;
        if (p.pin_d2) {
            const unsigned d2 = __ldg(p.pin_d2 + node);
            if (d2 != 255u) a += A_h(p, sqrtf((float)d2));
        }
        p.ah[node] = a;
    }
};

// Where the blocks of a near-contact launch come from. NcOne: one lattice, its
// parameters and tensor map in kernel parameter space. NcBatch: the lattices of a
// batch table (the serving engine's batched launches), global block b belonging to
// the last lattice whose first block is <= b; that lattice's parameters are copied to
// shared memory when the CTA takes the block. bind() is called by every thread of the
// CTA at the same point. Ghost tasks (the ghost copies of the step's input
// populations) are numbered over the whole launch.
struct NcOne {
    const StepParams* p;
    const CUtensorMap* map;
    int tma;
    __device__ __forceinline__ long long bind(long long b) { return b; }
    __device__ __forceinline__ const StepParams& params() const { return *p; }
    __device__ __forceinline__ const CUtensorMap* lag_map() const { return map; }
    __device__ __forceinline__ int tma_ok() const { return tma; }
    __device__ __forceinline__ long long ghost_total() const {
        return p->ghost_f ? ghost_work(*p) : 0;
    }
    template <class St>
    __device__ __forceinline__ void ghost(long long t, int lane) const {
        ghost_task<St>(static_cast<typename St::T*>(p->ghost_f), *p, t, lane);
    }
};
struct NcBatch {
    const NcBatchLattice* tab;
    int nlat;
    long long gtotal;
    StepParams* sp;   // in shared memory: the parameters of the lattice of the CTA's block
    int* lat;         // in shared memory: that lattice
    __device__ __forceinline__ long long bind(long long b) {
        __syncthreads();   // the previous block's parameters are no longer read
        if (threadIdx.x == 0) {
            int lo = 0, hi = nlat - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tab[mid].block_begin <= b) lo = mid;
                else hi = mid - 1;
            }
            *lat = lo;
        }
        __syncthreads();
        const int l = *lat;
        const int* src = reinterpret_cast<const int*>(&tab[l].p);
        int* dst = reinterpret_cast<int*>(sp);
        for (int i = threadIdx.x; i < (int)(sizeof(StepParams) / sizeof(int)); i += blockDim.x)
            dst[i] = src[i];
        __syncthreads();
        return b - tab[l].block_begin;
    }
    __device__ __forceinline__ const StepParams& params() const { return *sp; }
    __device__ __forceinline__ const CUtensorMap* lag_map() const { return &tab[*lat].lag_map; }
    __device__ __forceinline__ int tma_ok() const { return tab[*lat].tma_ok; }
    __device__ __forceinline__ long long ghost_total() const { return gtotal; }
    template <class St>
    __device__ __forceinline__ void ghost(long long t, int lane) const {
        int lo = 0, hi = nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].ghost_begin <= t) lo = mid;
            else hi = mid - 1;
        }
        const NcBatchLattice& L = tab[lo];
        if (L.p.ghost_f)
            ghost_task<St>(static_cast<typename St::T*>(L.p.ghost_f), L.p, t - L.ghost_begin, lane);
    }
};

// Work items of a lattice's near-contact pass: block columns x segments of nc_seg blocks.
__host__ __device__ inline long long nc_blocks(const StepParams& p) {
    const int seg = p.nc_seg > 0 ? p.nc_seg : 1, bzn = (p.nz + NB_Z - 1) / NB_Z;
    return (long long)((p.nx + NB_X - 1) / NB_X) * ((p.ny + NB_Y - 1) / NB_Y) *
           ((bzn + seg - 1) / seg);
}

// The pass over `nblocks` blocks of `src` (see nc_block_kernel below for what a block
// does); the CTA takes blocks blockIdx.x, + gridDim.x, ...
template <class St, int H, bool W, class Src>
__device__ __forceinline__ void nc_block_pass(Src& src, long long nitems, unsigned char* nsm) {
    using G = NcBlockGeo<H>;
    float* cube = reinterpret_cast<float*>(nsm);                           // [SZ][SY][SX]
    unsigned char* q = nsm + G::CUBE_BYTES;                                // 128-byte aligned
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(q);    // (4 slots, 1 used)
    int* rays = reinterpret_cast<int*>(q + 4 * sizeof(unsigned long long));   // [NB_NODES] listed nodes
    int* nrays = rays + NB_NODES;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // ghost tasks of this CTA: blockIdx.x + j gridDim.x for j = 0, 1, ...; a warp that
    // has no ray left in a block takes the next one (its scattered accesses then overlap
    // the other warps' rays), and all warps take the rest after the last block
    int* gnext = nrays + 3;
    if (tid == 0) *gnext = 0;
    __syncthreads();
    grid_dep_wait();
    const long long gtotal = src.ghost_total();
    auto ghost_next = [&]() {
        int j = 0;
        if (lane == 0) j = atomicAdd(gnext, 1);
        j = __shfl_sync(0xffffffffu, j, 0);
        const long long t = (long long)blockIdx.x + (long long)j * gridDim.x;
        if (t >= gtotal) return false;
        src.template ghost<St>(t, lane);
        return true;
    };
    uint32_t parity = 0u;
    bool failed = false;
    for (long long item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
        const long long li = src.bind(item);
        const StepParams& p = src.params();
        const size_t plane = (size_t)p.nx * p.ny;
        int bx, by, bz0, bz1;
        nc_item(p, li, bx, by, bz0, bz1);
        const int x0 = bx * NB_X, y0 = by * NB_Y;
        int zbase = 0;   // ring slot of the current block's first window plane
        for (int bz = bz0; bz < bz1; ++bz) {
            const int z0 = bz * NB_Z;
            // the first block of the segment copies its whole window, every later one the
            // NB_Z planes that enter it (into the slots of the planes that left); (a ring
            // slot's reads of the last block precede the copy into it: the barrier that
            // ended that block, then the proxy fence)
            fence_proxy_async();
            nc_fill_planes<H>(p, src.lag_map(), src.tma_ok(), x0, y0, z0, bz == bz0 ? 0 : G::SZ - NB_Z,
                              zbase, cube, bar);
            cp_async_wait<0>();
            // (a wait that gives up leaves its phase pending: the drain below waits on it)
            if (mbar_wait(bar, parity, p.err)) parity ^= 1u;
            else failed = true;
            if (__syncthreads_or(failed)) {
                failed = true;
                break;
            }
            // ---- 1. gradients and thresholds of the block's nodes: a node with |G'| >= 1e-3
            // and a first sample inside the fluid is listed; every other node's A_h is final
            // (0, or its pin term when it has a ray of no samples)
            if (tid == 0) *nrays = 0;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < NB_PER_THREAD; ++j) {
                const int idx = tid + j * NB_THREADS;
                const int lx = idx % NB_X, ly = (idx / NB_X) % NB_Y, lz = idx / (NB_X * NB_Y);
                const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
                bool listed = false;
                if (x < p.nx && y < p.ny && z < p.nz) {
                    float Gx, Gy, Gz, nx_, ny_, nz_;
                    cube_gradient<H, W>(p, cube, x, y, z, lx, ly, lz, zbase, Gx, Gy, Gz);
                    float a = 0.0f;
                    if (nc_ray(Gx, Gy, Gz, nx_, ny_, nz_)) {
                        listed = nc_sample_end(p, y, z, ny_, nz_) > 0;
                        if (!listed && p.pin_d2) {
                            const unsigned d2 = __ldg(p.pin_d2 + (size_t)z * plane + (size_t)y * p.nx + x);
                            if (d2 != 255u) a = A_h(p, sqrtf((float)d2));
                        }
                    }
                    if (!listed) p.ah[(size_t)z * plane + (size_t)y * p.nx + x] = a;
                }
                // (one atomic per warp)
                const unsigned m = __ballot_sync(0xffffffffu, listed);
                int base = 0;
                if (lane == 0 && m) base = atomicAdd(nrays, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (listed) rays[base + __popc(m & ((1u << lane) - 1u))] = idx;
            }
            __syncthreads();
            const int nr = *nrays;
            // ---- 2. the listed rays, one per thread: the sign class of every sample (all
            // rays of a lattice without walls have the same samples, so the lanes of a warp
            // stay together), then A_h from the sign masks and the samples around the two
            // crossings, interpolated again
            for (int k = tid; k < nr; k += NB_THREADS) {
                NcRay r;
                r.start<H, W>(p, cube, rays[k], x0, y0, z0, zbase);
                r.measure<H, W>(p, cube, y0, z0);
                r.finish(p, plane);
            }
            // (a warp without a ray in the last round: one ghost task)
            if ((tid & ~31) + NB_THREADS * ((nr + NB_THREADS - 1) / NB_THREADS - 1) >= nr || nr == 0)
                ghost_next();
            __syncthreads();   // the cube and the ray list are consumed
            zbase = ring_slot<H>(zbase, NB_Z);   // the next block's window starts NB_Z planes up
        }
    }
    if (failed) {
        // give a tensor copy still in flight into this CTA's cube a bounded chance to
        // land before the CTA exits
        for (uint32_t i = 0; i < (1u << 20); ++i)
            if (mbar_try_wait(bar, parity)) break;
    }
    cp_async_wait<0>();
    while (ghost_next()) {
    }
}

template <class St, int H, bool W>
__global__ void __launch_bounds__(NB_THREADS, 2)
nc_block_kernel(const StepParams p, const __grid_constant__ CUtensorMap lag_map, int tma_ok) {
    extern __shared__ __align__(128) unsigned char nsm[];
    if (threadIdx.x == 0)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&lag_map)) : "memory");
    NcOne src{&p, &lag_map, tma_ok};
    nc_block_pass<St, H, W>(src, nc_blocks(p), nsm);
    grid_dep_launch();
}

// The near-contact pass of every lattice of a batch table in one launch.
template <class St, int H>
__global__ void __launch_bounds__(NB_THREADS, 2)
nc_block_kernel_batched(const NcBatchLattice* __restrict__ tab, int nlat, long long nblocks,
                        long long ghost_total) {
    extern __shared__ __align__(128) unsigned char nsm[];
    __shared__ StepParams sp;
    __shared__ int lat;
    NcBatch src{tab, nlat, ghost_total, &sp, &lat};
    nc_block_pass<St, H, true>(src, nblocks, nsm);
}

// Launch with programmatic stream serialisation (see grid_dep_wait). (The list and
// ghost kernels keep the default shared-memory carveout: forcing the largest one
// leaves them less L1 and measured slower.)
template <class... KArgs, class... Args>
static cudaError_t pdl_launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class St, int H, bool W>
static cudaError_t launch_block_tpl(const StepParams& p, const CUtensorMap& lag_map, bool tma_ok,
                                   int num_sms, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(nc_block_kernel<St, H, W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)NcBlockGeo<H>::SMEM);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nc_block_kernel<St, H, W>,
                                                              NB_THREADS, NcBlockGeo<H>::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    return pdl_launch(nc_block_kernel<St, H, W>, (unsigned)(num_sms * per_sm), NB_THREADS,
                      NcBlockGeo<H>::SMEM, s, p, lag_map, tma_ok ? 1 : 0);
}

template <class St>
static cudaError_t launch_block_st(const StepParams& p, const CUtensorMap& lag_map, bool tma_ok,
                                   int num_sms, cudaStream_t s) {
    // halo: the farthest corner of a ray sample is floor(h_cut) + 3 nodes away
    const int need = (int)floorf(p.h_cut) + 3;
    // (lattices without walls take the instances without the wall tests)
    const bool w = p.wall_y || p.wall_z;
    if (need <= 9)
        return w ? launch_block_tpl<St, 9, true>(p, lag_map, tma_ok, num_sms, s)
                 : launch_block_tpl<St, 9, false>(p, lag_map, tma_ok, num_sms, s);
    if (need <= 12)
        return w ? launch_block_tpl<St, 12, true>(p, lag_map, tma_ok, num_sms, s)
                 : launch_block_tpl<St, 12, false>(p, lag_map, tma_ok, num_sms, s);
    return cudaErrorInvalidValue;   // h_cut <= 9 is checked when the context is made
}

cudaError_t launch_nc_block(const StepParams& p, const CUtensorMap& lag_map, bool tma_ok,
                            int storage, int num_sms, cudaStream_t s) {
    // (the pass touches populations only in the ghost fill, which depends on the
    // element type alone: the reduced form shares the FP32 instance)
    switch (storage) {
        case 0: case 3: return launch_block_st<StoreF32>(p, lag_map, tma_ok, num_sms, s);
        case 1: case 4: return launch_block_st<StoreF16>(p, lag_map, tma_ok, num_sms, s);
        case 2: return launch_block_st<StoreBF16>(p, lag_map, tma_ok, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

template <class St, int H>
static cudaError_t launch_block_batched_tpl(const NcBatchLattice* tab, int nlat, long long nblocks,
                                           long long ghost_total, int num_sms, cudaStream_t s) {
    static int per_sm = 0;
    if (!tab) {   // preparation only: the shared-memory attribute, outside stream capture
        cudaError_t e = cudaFuncSetAttribute(nc_block_kernel_batched<St, H>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)NcBlockGeo<H>::SMEM);
        if (e == cudaSuccess && per_sm == 0)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nc_block_kernel_batched<St, H>,
                                                              NB_THREADS, NcBlockGeo<H>::SMEM);
        return e;
    }
    const long long g = std::min<long long>((long long)num_sms * std::max(1, per_sm),
                                            std::max<long long>(1, nblocks));
    nc_block_kernel_batched<St, H><<<(unsigned)g, NB_THREADS, NcBlockGeo<H>::SMEM, s>>>(
        tab, nlat, nblocks, ghost_total);
    return cudaGetLastError();
}

template <class St>
static cudaError_t launch_block_batched_st(const NcBatchLattice* tab, int nlat, long long nblocks,
                                          long long ghost_total, double h_cut, int num_sms,
                                          cudaStream_t s) {
    const int need = (int)std::floor(h_cut) + 3;
    if (need <= 9) return launch_block_batched_tpl<St, 9>(tab, nlat, nblocks, ghost_total, num_sms, s);
    if (need <= 12) return launch_block_batched_tpl<St, 12>(tab, nlat, nblocks, ghost_total, num_sms, s);
    return cudaErrorInvalidValue;
}

// The near-contact pass of every lattice of a batch table (one storage element type and
// one halo depth, i.e. h_cut class) in one launch.
cudaError_t launch_nc_batched(const NcBatchLattice* tab, int nlat, long long nblocks,
                              long long ghost_total, int storage, double h_cut, int num_sms,
                              cudaStream_t s) {
    switch (storage) {
        case 0: case 3:
            return launch_block_batched_st<StoreF32>(tab, nlat, nblocks, ghost_total, h_cut, num_sms, s);
        case 1: case 4:
            return launch_block_batched_st<StoreF16>(tab, nlat, nblocks, ghost_total, h_cut, num_sms, s);
        case 2:
            return launch_block_batched_st<StoreBF16>(tab, nlat, nblocks, ghost_total, h_cut, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

// Shared-memory attribute of the batched near-contact kernel of one storage element
// type and halo class: set before any launch (and outside stream capture).
cudaError_t prepare_nc_batched(int storage, double h_cut) {
    return launch_nc_batched(nullptr, 0, 0, 0, storage, h_cut, 1, nullptr);
}

// Halo class of a near-contact pass (lattices sharing it can be batched).
int nc_halo(double h_cut) {
    const int need = (int)std::floor(h_cut) + 3;
    return need <= 9 ? 9 : 12;
}

// Blocks of nodes of a lattice's near-contact pass.
long long nc_block_count(const StepParams& p) { return nc_blocks(p); }

// Shape of the box a tensor copy of the near-contact pass fills (x, y, z extents: one
// plane of a halo cube), for the tensor map of a colour field.
void nc_cube_box(double h_cut, int box[3]) {
    const int need = (int)std::floor(h_cut) + 3;
    const int H = need <= 9 ? 9 : 12;
    const int HX = (H + 3) / 4 * 4;
    box[0] = NB_X + 2 * HX;
    box[1] = NB_Y + 2 * H;
    box[2] = 1;
}

// Blocks per z segment of a block column in the near-contact pass: up to 16 (a block's
// window shares all but NB_Z of its planes with the last one's), fewer where the
// lattice has too few columns for about four work items per CTA (two CTAs per SM).
int nc_segment_blocks(int nx, int ny, int nz, int num_sms) {
    const long long cols = (long long)((nx + NB_X - 1) / NB_X) * ((ny + NB_Y - 1) / NB_Y);
    const long long bzn = (nz + NB_Z - 1) / NB_Z;
    const long long want = 8LL * std::max(1, num_sms);
    return (int)std::max<long long>(1, std::min<long long>({16LL, bzn, cols * bzn / want}));
}

template <class St, bool U, bool SC>
static cudaError_t launch_tpl3(const StepParams& p, const CUtensorMap& map,
                               const CUtensorMap& omap, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<St, U, SC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Geo<St, SC>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return pdl_launch(step_kernel<St, U, SC>, (unsigned)grid, NT, Geo<St, SC>::SMEM, s, p, map,
                      omap);
}

// omega == 1 everywhere (equal relaxation times tau = 1) drops the non-equilibrium
// terms of the collision
template <class St>
static cudaError_t launch_tpl(const StepParams& p, const CUtensorMap& map, const CUtensorMap& omap,
                              int grid, cudaStream_t s) {
    const bool unit = !p.var_tau && p.omega0 == 1.0f;
    if constexpr (St::RED) {
        if (p.model == 1) return cudaErrorInvalidValue;   // refused when the context is made
    } else {
        if (p.model == 1)
            return unit ? launch_tpl3<St, true, true>(p, map, omap, grid, s)
                        : launch_tpl3<St, false, true>(p, map, omap, grid, s);
    }
    return unit ? launch_tpl3<St, true, false>(p, map, omap, grid, s)
                : launch_tpl3<St, false, false>(p, map, omap, grid, s);
}

cudaError_t launch_step(const StepParams& p, const CUtensorMap& map, const CUtensorMap& omap,
                        int storage, int grid, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_tpl<StoreF32>(p, map, omap, grid, s);
        case 1: return launch_tpl<StoreF16>(p, map, omap, grid, s);
        case 2: return launch_tpl<StoreBF16>(p, map, omap, grid, s);
        case 3: return launch_tpl<StoreQ5>(p, map, omap, grid, s);
        case 4: return launch_tpl<StoreQ5H>(p, map, omap, grid, s);
    }
    return cudaErrorInvalidValue;
}

template <class St>
static cudaError_t launch_aa_tpl(const StepParams& p, int layout, int num_sms, cudaStream_t s) {
    // a grid that fills the GPU once (CTAs loop over the row segments)
    static int per_sm[2] = {0, 0};
    const bool unit = !p.var_tau && p.omega0 == 1.0f;
    auto collide = unit ? aa_collide_kernel<St, true> : aa_collide_kernel<St, false>;
    if (per_sm[unit] == 0) {
        int a = 0, b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, aa_phi_kernel<St>, AA_W, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, collide, AA_W, 0);
        if (e != cudaSuccess) return e;
        per_sm[unit] = std::max(1, std::min(a, b));
    }
    const long long items = aa_items(p);
    const unsigned grid = (unsigned)std::max(1LL, std::min(items, (long long)num_sms * per_sm[unit]));
    cudaError_t e = pdl_launch(aa_phi_kernel<St>, grid, AA_W, 0, s, p, layout);
    if (e != cudaSuccess) return e;
    return pdl_launch(collide, grid, AA_W, 0, s, p, layout);
}

// One in-place step from state layout `layout` (p.fin == p.fout: the one copy).
cudaError_t launch_aa_step(const StepParams& p, int layout, int storage, int num_sms,
                           cudaStream_t s) {
    switch (storage) {
        case 0: return launch_aa_tpl<StoreF32>(p, layout, num_sms, s);
        case 1: return launch_aa_tpl<StoreF16>(p, layout, num_sms, s);
        case 2: return launch_aa_tpl<StoreBF16>(p, layout, num_sms, s);
    }
    return cudaErrorInvalidValue;   // the reduced forms are not stored in place
}

template <class St, bool U, bool SC>
static cudaError_t launch_batched_tpl(const BatchLattice* tab, int nlat, int ctas, cudaStream_t s) {
    step_kernel_batched<St, U, SC><<<ctas, NT, Geo<St, SC>::SMEM, s>>>(tab, nlat);
    return cudaGetLastError();
}

template <class St, bool U, bool SC>
static cudaError_t prepare_batched_tpl() {
    return cudaFuncSetAttribute(step_kernel_batched<St, U, SC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<St, SC>::SMEM);
}

// Batched kernel of one (storage, relaxation class, model): dispatched over the
// 16 combinations (the reduced forms hold no Shan-Chen state) with a callable that
// takes the three as template arguments.
template <class F>
static cudaError_t batched_dispatch(int storage, bool unit_omega, int model, F&& fn) {
    const bool sc = model == 1;
    switch (storage * 4 + (unit_omega ? 2 : 0) + (sc ? 1 : 0)) {
        case 0: return fn.template operator()<StoreF32, false, false>();
        case 1: return fn.template operator()<StoreF32, false, true>();
        case 2: return fn.template operator()<StoreF32, true, false>();
        case 3: return fn.template operator()<StoreF32, true, true>();
        case 4: return fn.template operator()<StoreF16, false, false>();
        case 5: return fn.template operator()<StoreF16, false, true>();
        case 6: return fn.template operator()<StoreF16, true, false>();
        case 7: return fn.template operator()<StoreF16, true, true>();
        case 8: return fn.template operator()<StoreBF16, false, false>();
        case 9: return fn.template operator()<StoreBF16, false, true>();
        case 10: return fn.template operator()<StoreBF16, true, false>();
        case 11: return fn.template operator()<StoreBF16, true, true>();
        case 12: return fn.template operator()<StoreQ5, false, false>();
        case 14: return fn.template operator()<StoreQ5, true, false>();
        case 16: return fn.template operator()<StoreQ5H, false, false>();
        case 18: return fn.template operator()<StoreQ5H, true, false>();
    }
    return cudaErrorInvalidValue;
}

struct PrepareBatched {
    template <class St, bool U, bool SC>
    cudaError_t operator()() const { return prepare_batched_tpl<St, U, SC>(); }
};
struct LaunchBatched {
    const BatchLattice* tab;
    int nlat, ctas;
    cudaStream_t s;
    template <class St, bool U, bool SC>
    cudaError_t operator()() const { return launch_batched_tpl<St, U, SC>(tab, nlat, ctas, s); }
};

// Shared-memory attribute of a batched step kernel: set before any launch (and
// outside stream capture).
cudaError_t prepare_step_batched(int storage, bool unit_omega, int model) {
    return batched_dispatch(storage, unit_omega, model, PrepareBatched{});
}

// One launch advancing every lattice of a device table by one step (all lattices of
// one storage format, relaxation class and model).
cudaError_t launch_step_batched(const BatchLattice* tab, int nlat, int ctas, int storage,
                                bool unit_omega, int model, cudaStream_t s) {
    return batched_dispatch(storage, unit_omega, model, LaunchBatched{tab, nlat, ctas, s});
}

cudaError_t launch_ghost_batched(const BatchLattice* tab, int nlat, long long cells, int storage,
                                 int num_sms, cudaStream_t s) {
    long long blocks = (cells + 7) / 8;   // a warp per task, 8 warps per block
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    if (blocks < 1) blocks = 1;
    switch (storage) {
        case 0: case 3: ghost_fill_batched<StoreF32><<<(unsigned)blocks, 256, 0, s>>>(tab, nlat, cells); break;
        case 1: case 4: ghost_fill_batched<StoreF16><<<(unsigned)blocks, 256, 0, s>>>(tab, nlat, cells); break;
        case 2: ghost_fill_batched<StoreBF16><<<(unsigned)blocks, 256, 0, s>>>(tab, nlat, cells); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Warp tasks of one lattice's ghost fill.
long long ghost_cells(const StepParams& p) { return ghost_work(p); }

template <class St>
static cudaError_t launch_ghost_tpl(void* f, const StepParams& p, unsigned blocks, unsigned threads,
                                   cudaStream_t s) {
    return pdl_launch(ghost_fill_kernel<St>, blocks, threads, 0, s,
                      static_cast<typename St::T*>(f), p);
}

cudaError_t launch_ghost_fill(void* f, const StepParams& p, int storage, int num_sms,
                              cudaStream_t s) {
    const int threads = 256;
    const size_t cells = (size_t)ghost_work(p);
    if (cells == 0) return cudaSuccess;   // nothing to copy (no launch)
    size_t blocks = (cells + threads / 32 - 1) / (threads / 32);   // a warp per task
    const size_t cap = (size_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    switch (storage) {
        case 0: case 3: return launch_ghost_tpl<StoreF32>(f, p, (unsigned)blocks, threads, s);
        case 1: case 4: return launch_ghost_tpl<StoreF16>(f, p, (unsigned)blocks, threads, s);
        case 2: return launch_ghost_tpl<StoreBF16>(f, p, (unsigned)blocks, threads, s);
    }
    return cudaErrorInvalidValue;
}

// Geometry the host needs for the tensor maps.
int step_tile_x() { return TX; }
int step_tile_y() { return TY; }
int step_box_rows() { return SH; }
int step_box_width(int storage) {
    return (storage == 0 || storage == 3) ? Geo<StoreF32>::BW : Geo<StoreF16>::BW;
}
int step_pad_x(int storage) {
    return (storage == 0 || storage == 3) ? Geo<StoreF32>::PADX : Geo<StoreF16>::PADX;
}
int step_ctas_per_sm() { return CTAS_PER_SM; }

}  // namespace lbm
