// lbm_step.cu -- the fused time-step kernel (one launch = one full lattice update).
//
// Data layout: populations in [2 species][19 directions][z][y][x] (x fastest), two
// copies (read one, write the other).
//
// A CTA owns a 32 x 16 tile of (x, y) columns and marches along z. For every plane p
// it stages in shared memory, per species and direction i, the rows of the source
// plane p - c_iz that the pull of the tile and of a one-node ring around it reads
// (rows y0-1-c_iy .. y0+16-c_iy, columns x0-PAD .. x0+32+PAD). Rows are moved with
// cp.async.bulk (16-byte aligned bulk copies, wrapped rows split in two) that
// complete on an mbarrier, two planes in flight. From a staged plane every thread
// pulls its node with constant-offset shared-memory loads, the colour field of the
// plane (tile + ring) goes to a 4-slot ring buffer, and one plane behind, the owned
// nodes are collided using the isotropic gradient read from that ring. The colour
// field of the same step is thus available at all 18 neighbours without a second
// pass over the populations. Links whose source lies beyond a bounce-back wall read
// the node's own opposite population directly from global memory.
//
// Work split: z is cut into `zparts` equal parts and every CTA marches one part of
// one tile. CTAs are numbered part-major, so the CTAs resident at the same time work
// on neighbouring tiles at the same heights: the halo rows one tile stages are the
// rows its neighbours are reading, and come from L2 rather than HBM.
// Lattices whose x extent is not a multiple of 32 (or that need element-wise
// wrapping) stage rows with ordinary loads instead of bulk copies; the compute is
// identical, so results do not depend on the staging path.
#include "lbm_device.cuh"

namespace lbm {

constexpr int TX = 32, TY = 16, NT = TX * TY;
constexpr int SH = TY + 2, SWP = TX + 2;   // colour-field ring: rows, columns
constexpr int NRING = 2 * (TX + 2) + 2 * TY;

template <class St>
struct Geo {
    using T = typename St::T;
    static constexpr int PAD = 16 / (int)sizeof(T);       // 16-byte alignment of rows
    static constexpr int W = TX + 2 * PAD;                  // staged row length (elements)
    static constexpr int ROWS = 2 * Q * SH;                 // staged rows per plane
    static constexpr size_t STAGE_BYTES = (size_t)ROWS * W * sizeof(T);
    static constexpr size_t PHI_BYTES = 4 * SH * SWP * sizeof(float);
    static constexpr size_t SMEM = 2 * STAGE_BYTES + PHI_BYTES + 2 * sizeof(unsigned long long);
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
    mbar_expect_tx(bar, bytes);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on an mbarrier phase: gives up after ~2^24 polls, records the failure
// in the error word and returns false (the caller then stops).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int* err) {
    for (uint32_t it = 0; it < (1u << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
}

// ---------------------------------------------------------------- the kernel
template <class St>
__global__ void __launch_bounds__(NT, 1) step_kernel(const StepParams p) {
    using T = typename St::T;
    using G = Geo<St>;
    constexpr int W = G::W, PAD = G::PAD;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage0 = reinterpret_cast<T*>(smem);
    float* sphi = reinterpret_cast<float*>(smem + 2 * G::STAGE_BYTES);   // [4][SH][SWP]
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(smem + 2 * G::STAGE_BYTES + G::PHI_BYTES);

    const T* __restrict__ fin = static_cast<const T*>(p.fin);
    T* __restrict__ fout = static_cast<T*>(p.fout);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const size_t plane = (size_t)p.nx * p.ny;

    if (tid == 0) {
        mbar_init(&bars[0], NT);
        mbar_init(&bars[1], NT);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    bool failed = false;

    // one (z part, tile) work item per CTA, part-major
    const int ntiles = p.tiles_x * p.tiles_y;
    const int part = blockIdx.x / ntiles, tile = blockIdx.x - part * ntiles;
    {
        const int zb = (int)((long long)p.nz * part / p.zparts);
        const int ze = (int)((long long)p.nz * (part + 1) / p.zparts);
        const int x0 = (tile % p.tiles_x) * TX, y0 = (tile / p.tiles_x) * TY;
        const int xw = min(TX, p.nx - x0), yh = min(TY, p.ny - y0);   // owned extent
        const bool fast = p.bulk_ok;   // aligned bulk-copy staging possible

        // ---- this thread's owned node and (optionally) one ring node
        const int otx = lane, oty = warp;
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

        // ---- staging of plane pl into buffer b (rows of every species/direction)
        auto issue = [&](int b, int pl) {
            T* st = stage0 + (size_t)b * (G::ROWS * W);
            const bool pvalid = !failed && (!p.wall_z || (pl >= 0 && pl < p.nz));
            if (pvalid) {
                for (int row = tid; row < G::ROWS; row += NT) {
                    const int ik = row / SH, r = row - ik * SH;
                    const int i = ik < Q ? ik : ik - Q;
                    const int zs0 = pl - cz(i);
                    const int ys0 = y0 - 1 - cy(i) + r;
                    if ((p.wall_z && (zs0 < 0 || zs0 >= p.nz)) || (p.wall_y && (ys0 < 0 || ys0 >= p.ny)))
                        continue;
                    const int zs = wrapi(zs0, p.nz), ys = wrapi(ys0, p.ny);
                    const T* src = fin + (size_t)ik * p.N + (size_t)zs * plane + (size_t)ys * p.nx;
                    T* dst = st + (size_t)row * W;
                    if (fast) {
                        // columns x0-PAD .. x0+TX+PAD-1, wrapped at 0 and nx in whole pieces
                        int xa = x0 - PAD, c = 0;
                        if (xa < 0) {
                            bulk_g2s(dst, src + (p.nx + xa), (uint32_t)(-xa * sizeof(T)), &bars[b]);
                            c = -xa;
                            xa = 0;
                        }
                        int len = min(W - c, p.nx - xa);
                        bulk_g2s(dst + c, src + xa, (uint32_t)(len * sizeof(T)), &bars[b]);
                        c += len;
                        if (c < W) {
                            bulk_g2s(dst + c, src, (uint32_t)((W - c) * sizeof(T)), &bars[b]);
                        }
                    } else {
                        // element-wise: only the columns the pulls read (PAD-2 .. TX+PAD+1)
                        for (int c = PAD - 2; c < TX + PAD + 2; ++c)
                            dst[c] = src[wrapi(x0 - PAD + c, p.nx)];
                    }
                }
            }
            mbar_arrive(&bars[b]);
        };
        auto wait = [&](int b) {
            if (!failed && !mbar_wait(&bars[b], parity[b], p.err)) failed = true;
            parity[b] ^= 1u;
        };

        // ---- pull of node (tx, ty) of plane pl from staged buffer b
        // returns densities; for keep == true also the total populations
        auto pull = [&](int b, int pl, int tx, int ty, float (&ft)[Q], float& rr, float& rb,
                        bool keep) {
            const T* st = stage0 + (size_t)b * (G::ROWS * W) + (size_t)(ty + 1) * W + (tx + PAD);
            const int gy = y0 + ty;
            const bool ylo = p.wall_y && gy == 0, yhi = p.wall_y && gy == p.ny - 1;
            const bool zlo = p.wall_z && pl == 0, zhi = p.wall_z && pl == p.nz - 1;
            const bool any_wall = ylo || yhi || zlo || zhi;
            float vr[Q], vb[Q];
            const float refh = p.ref_half;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float ref = wgt(i) * refh;
                vr[i] = St::cvt(st[(size_t)i * SH * W - cx(i)], ref);
                vb[i] = St::cvt(st[(size_t)(Q + i) * SH * W - cx(i)], ref);
            }
            if (any_wall) {
                const size_t self = (size_t)pl * plane + (size_t)wrapi(gy, p.ny) * p.nx + wrapi(x0 + tx, p.nx);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const bool out = (cy(i) > 0 && ylo) || (cy(i) < 0 && yhi) ||
                                     (cz(i) > 0 && zlo) || (cz(i) < 0 && zhi);
                    if (out) {
                        const float ref = wgt(i) * refh;
                        vr[i] = St::load(fin, (size_t)opp(i) * p.N + self, ref);
                        vb[i] = St::load(fin, (size_t)(Q + opp(i)) * p.N + self, ref);
                    }
                }
            }
            rr = sum19(vr);
            rb = sum19(vb);
            if (keep) {
#pragma unroll
                for (int i = 0; i < Q; ++i) ft[i] = vr[i] + vb[i];
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
            const int plw = wrapi(pl, p.nz);
            if (owned) {
                pull(b, plw, otx, oty, ft, rr, rb, keep);
                phi_at(slot(pl), otx, oty) = (rr - rb) / (rr + rb);
            }
            if (ring) {
                float dummy[Q], a, c;
                pull(b, plw, rtx, rty, dummy, a, c, false);
                phi_at(slot(pl), rtx, rty) = (a - c) / (a + c);
            }
        };

        float cur[Q], nxt[Q];
        float c_rr = 0.f, c_rb = 0.f, n_rr = 0.f, n_rb = 0.f;

        // ---- prologue: planes zb-1 and zb
        fence_proxy_async();
        issue(0, zb - 1);
        issue(1, zb);
        wait(0);
        densities(0, zb - 1, nxt, n_rr, n_rb, false);
        __syncthreads();
        fence_proxy_async();
        issue(0, zb + 1);
        wait(1);
        densities(1, zb, cur, c_rr, c_rb, true);
        __syncthreads();

        for (int z = zb; z < ze; ++z) {
            const int bn = (z + 1 - zb + 1) & 1;   // buffer of plane z+1
            fence_proxy_async();
            if (z + 2 <= ze) issue(bn ^ 1, z + 2);
            wait(bn);
            densities(bn, z + 1, nxt, n_rr, n_rb, true);
            __syncthreads();
            if (owned && !failed) {
                const int x = x0 + otx, y = y0 + oty;
                const bool ylo = p.wall_y && y == 0, yhi = p.wall_y && y == p.ny - 1;
                const bool zlo = p.wall_z && z == 0, zhi = p.wall_z && z == p.nz - 1;
                const float phic = phi_at(slot(z), otx, oty);
                // isotropic colour gradient, 3 w_i = 1/6 (faces), 1/12 (edges); a
                // neighbour beyond a wall takes the centre value
                float Gx = 0.f, Gy = 0.f, Gz = 0.f;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (i == 9) continue;
                    const bool wall = (cy(i) < 0 && ylo) || (cy(i) > 0 && yhi) ||
                                      (cz(i) < 0 && zlo) || (cz(i) > 0 && zhi);
                    const float v = wall ? phic : phi_at(slot(z + cz(i)), otx + cx(i), oty + cy(i));
                    const float w3 = csq(i) == 1 ? (1.0f / 6.0f) : (1.0f / 12.0f);
                    if (cx(i)) Gx += (cx(i) > 0 ? w3 : -w3) * v;
                    if (cy(i)) Gy += (cy(i) > 0 ? w3 : -w3) * v;
                    if (cz(i)) Gz += (cz(i) > 0 ? w3 : -w3) * v;
                }
                const size_t node = (size_t)z * plane + (size_t)y * p.nx + x;
                float Fx = __ldg(p.fx_row + y), Fy = p.gy, Fz = p.gz;
                if (p.A_nc > 0.0f) {
                    // near-contact force A_h G, A_h measured by the near-contact pass;
                    // the entry is consumed (reset to 0) so that only the next pass's
                    // candidates are nonzero when the next step reads it
                    const float ah = p.ah[node];
                    if (ah != 0.0f) {
                        Fx += ah * Gx;
                        Fy += ah * Gy;
                        Fz += ah * Gz;
                        p.ah[node] = 0.0f;
                    }
                    // this node's gradient is the next pass's lagged gradient: list it
                    // as a candidate if it may reach the 1e-3 threshold there
                    const bool cand = Gx * Gx + Gy * Gy + Gz * Gz >= 0.81e-6f;
                    const unsigned m = __ballot_sync(__activemask(), cand);
                    if (cand) {
                        const int leader = __ffs(m) - 1;
                        int base = 0;
                        if (lane == leader) base = atomicAdd(p.cand_count, __popc(m));
                        base = __shfl_sync(m, base, leader);
                        p.cand[base + __popc(m & ((1u << lane) - 1u))] = (int)node;
                    }
                }
                collide_store<St>(p, cur, c_rr, c_rb, Gx, Gy, Gz, Fx, Fy, Fz, fout, node);
                p.phi_out[node] = phic;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
            c_rr = n_rr;
            c_rb = n_rb;
        }
    }
    if (failed) {
        // give copies still in flight into this CTA's shared memory a bounded chance
        // to land before the CTA exits
        for (int b = 0; b < 2; ++b)
            for (uint32_t it = 0; it < (1u << 20); ++it)
                if (mbar_try_wait(&bars[b], parity[b])) break;
    }
}

// ---------------------------------------------------------------- near-contact pass
// A_h from the lagged colour field. In list mode it visits only the candidate nodes
// the previous step kernel listed (lagged gradient >= 0.9e-3, a superset of the
// nodes where A_h can be nonzero), one thread per node, so rays do not diverge
// across a warp with non-interface lanes. In scan mode (first step after the state
// was set) each block takes 1024 consecutive nodes, writes 0 everywhere, gathers
// the candidates into a shared-memory list and marches their rays.
constexpr int NC_THREADS = 256, NC_CHUNK = 1024;

__global__ void __launch_bounds__(NC_THREADS) nc_kernel(const StepParams p) {
    __shared__ int list[NC_CHUNK];
    __shared__ int count;
    const size_t N = p.N;
    const size_t plane = (size_t)p.nx * p.ny;
    if (p.nc_list) {
        // list mode: the candidates written by the previous step kernel (every other
        // entry of ah is 0, consumed by that kernel)
        const int cnt = *p.nc_count;
        for (int k = blockIdx.x * NC_THREADS + threadIdx.x; k < cnt; k += gridDim.x * NC_THREADS) {
            const size_t n = (size_t)p.nc_list[k];
            const int z = (int)(n / plane);
            const int rem = (int)(n - (size_t)z * plane);
            const int y = rem / p.nx, x = rem - y * p.nx;
            const float a = nc_strength(p, n, x, y, z);
            if (a != 0.0f) p.ah[n] = a;
        }
        return;
    }
    // scan mode: every node
    for (size_t base = (size_t)blockIdx.x * NC_CHUNK; base < N; base += (size_t)gridDim.x * NC_CHUNK) {
        if (threadIdx.x == 0) count = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < NC_CHUNK; k += NC_THREADS) {
            const size_t n = base + k;
            if (n >= N) break;
            const int z = (int)(n / plane);
            const int rem = (int)(n - (size_t)z * plane);
            const int y = rem / p.nx, x = rem - y * p.nx;
            float Gx, Gy, Gz;
            gradient_global(p, p.phi_lag, x, y, z, Gx, Gy, Gz);
            if (Gx * Gx + Gy * Gy + Gz * Gz >= 0.81e-6f) list[atomicAdd(&count, 1)] = k;
            p.ah[n] = 0.0f;
        }
        __syncthreads();
        const int cnt = count;
        for (int k = threadIdx.x; k < cnt; k += NC_THREADS) {
            const size_t n = base + list[k];
            const int z = (int)(n / plane);
            const int rem = (int)(n - (size_t)z * plane);
            const int y = rem / p.nx, x = rem - y * p.nx;
            p.ah[n] = nc_strength(p, n, x, y, z);
        }
        __syncthreads();
    }
}

cudaError_t launch_nc(const StepParams& p, int num_sms, cudaStream_t s) {
    size_t blocks = (p.N + NC_CHUNK - 1) / NC_CHUNK;
    const size_t cap = (size_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    nc_kernel<<<(unsigned)blocks, NC_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

template <class St>
static cudaError_t launch_tpl(const StepParams& p, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Geo<St>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    step_kernel<St><<<grid, NT, Geo<St>::SMEM, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepParams& p, int storage, int grid, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_tpl<StoreF32>(p, grid, s);
        case 1: return launch_tpl<StoreF16>(p, grid, s);
        case 2: return launch_tpl<StoreBF16>(p, grid, s);
    }
    return cudaErrorInvalidValue;
}

int step_tile_x() { return TX; }
int step_tile_y() { return TY; }

}  // namespace lbm
