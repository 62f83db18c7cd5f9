/*
 * lbm.h -- C-ABI of the GB300 (sm_103a) library liblbm.so: one time step of the
 * two-component colour-gradient lattice Boltzmann method on the D3Q19 lattice
 * (Succi et al., "Towards Exascale Design of Soft Mesoscale Materials",
 * arXiv:2005.12764, Secs. "Basics of Lattice Boltzmann Method", "Multi-component
 * flows" and "LB method for microfluidic crystals").
 *
 * One step (lbm_step) is, for every node, in this order:
 *   pull streaming with halfway bounce-back walls       Eq. (1) and the streaming text
 *   moments rho_r, rho_b, j, colour field phi            Eq. (3)
 *   isotropic colour gradient G = 3 sum_i w_i c_i phi(x+c_i)   stencil form of Eq. (10)
 *   force F = body + Kolmogorov + near-contact            Eq. (11)
 *   BGK of the total population + EDM source              Eqs. (1), (2), (5)-(9)
 *   colour-gradient perturbation (surface tension sigma)  generalised perturbation
 *   recolouring of the two species (segregation beta)     Latva-Kokko & Rothman
 * The last two steps are not written in the paper; the library implements the
 * published colour-gradient method it cites, as documented below.
 *
 * Conventions shared by every entry point:
 *  - Lattice nx*ny*nz nodes, node index n = (z*ny + y)*nx + x (x fastest).
 *  - Fields passed in or out are float64 arrays: scalar fields [N], vector fields
 *    [3][N] (component-major). Host pointers when on_device == 0; CUDA device
 *    pointers (e.g. torch.Tensor.data_ptr()) on the same device when on_device == 1.
 *    The caller owns every array; the library copies what it needs.
 *  - Work is queued on the context's CUDA stream (params.cuda_stream, NULL = the
 *    legacy default stream). Calls that return data to the host synchronise that
 *    stream; lbm_step does not.
 *  - Errors are reported by return code, never by exceptions or aborts.
 *    lbm_last_error() gives a message. After LBM_ECUDA the context should be
 *    destroyed; after any other error it stays usable.
 *  - A context is not thread-safe: use one context per host thread and stream.
 *  - All arithmetic of the step is FP32; FP64 is used only for the set/get
 *    conversions and the conservation / Laplace reductions.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,   /* bad argument or parameter; nothing was changed          */
    LBM_ENOMEM = -2,   /* device or host allocation failed                         */
    LBM_ECUDA = -3,    /* a CUDA call failed; destroy the context                  */
    LBM_ESTATE = -4,   /* call out of order (e.g. lbm_step before lbm_set_fields)  */
    LBM_ETIMEOUT = -5  /* a bounded device-side wait gave up                       */
} lbm_status;

/* Storage of the populations in device memory. Arithmetic is FP32 in all cases.
 * FP16/BF16 store, rounded to nearest even, the deviation of f_i^k from
 * w_i rho0 (1 + s_k phi)/2 (s_r = +1, s_b = -1), where phi is the colour field of
 * the node that wrote the population, in the step that wrote it: the species'
 * share of the reference rest population w_i rho0 of the total population:
 * the total deviation f_i - w_i rho0 split between the species by colour.
 *
 * LBM_STORE_FP32_Q5 is an exact reduced FP32 form of the colour-gradient state:
 * Q + 5 values per node instead of 2Q (192 instead of 304 bytes moved per node and
 * step). After recolouring, the two species' populations of a node are
 *   f^r_i = kappa_r f_i + w_i (c_i . m)/|c_i|,  f^b_i = kappa_b f_i - w_i (c_i . m)/|c_i|,
 * f_i = f^r_i + f^b_i, kappa_k = rho_k/rho, m = beta (rho_r rho_b/rho) n with n the
 * unit colour gradient (m = 0 where the gradient vanishes). The form stores the 19
 * totals f_i and (kappa_r, kappa_b, m); each streamed population is split with the
 * coefficients of the node it comes from. The Shan-Chen model is refused with it
 * (its species do not share one population). lbm_get_pops returns the rebuilt
 * species populations; lbm_set_pops stores a split of the recoloured form exactly
 * and projects any other split onto that form (kappa_k from the species sums, m
 * from the first moment of f^r_i - kappa_r f_i).
 *
 * LBM_STORE_FP16_Q5 is the same reduced form with the 19 totals stored in FP16 as
 * deviations f_i - w_i rho0 from the lattice weights (rounded to nearest even; the
 * total density is close to rho0 in both phases, so the deviation is small), and the
 * five coefficients kept exact in FP32 (each as two 16-bit arrays: the low and the
 * high half of its bits), so that the species masses they carry are not rounded:
 * 2 x (19 x 2 + 5 x 4) = 116 bytes moved per node and step. All arithmetic is FP32,
 * as in every form.                                                                */
typedef enum {
    LBM_STORE_FP32 = 0,
    LBM_STORE_FP16_DEV = 1,
    LBM_STORE_BF16_DEV = 2,
    LBM_STORE_FP32_Q5 = 3,
    LBM_STORE_FP16_Q5 = 4
} lbm_storage;

/* Binary-mixture model (Sec. "Multi-component flows"). LBM_MODEL_COLOUR: the
 * colour-gradient model (BGK of the total population + EDM source, perturbation,
 * recolouring, optional near-contact force). LBM_MODEL_SHAN_CHEN: each species
 * relaxes at the mixture rate towards f^eq(rho_k, u), u = j/rho, with the EDM
 * source of its own force F^k = -G_sc rho_k sum_i w_i rho_kbar(x + c_i) c_i
 * (Eq. (12), with the sign that makes G_sc > 0 repulsive, as the text states) plus
 * its share rho_k/rho of the body force; sigma, beta are unused and A_nc must be 0.
 * A neighbour beyond a wall takes the node's own densities in either model.      */
typedef enum { LBM_MODEL_COLOUR = 0, LBM_MODEL_SHAN_CHEN = 1 } lbm_model;

typedef struct {
    int nx, ny, nz;          /* lattice size, each >= 1                                  */
    int wall_y, wall_z;      /* 1 = halfway bounce-back walls at y (z) = -1/2 and n-1/2;
                                0 = periodic. x is always periodic.                      */
    double tau_r, tau_b;     /* relaxation times (> 1/2) of the red and blue species;
                                nu_k = (tau_k - 1/2)/3, Eq. (4). The mixture relaxes at
                                omega = 2c_s^2/(2 nu + c_s^2) with 1/nu the density-
                                weighted mean of 1/nu_k, Eqs. (7)-(8) (Eq. (7) read with
                                a plus sign, consistent with Eq. (4)).                   */
    double sigma;            /* surface tension; perturbation amplitude A = 9 omega sigma/2 */
    double beta;             /* recolouring segregation parameter in [0, 1]               */
    double A_nc;             /* near-contact amplitude A of Eq. (11); 0 = off             */
    double h_min;            /* plateau length of A_h[h] (lattice units), e.g. 3          */
    double h_cut;            /* cutoff of A_h[h]; <= 0 means 2*h_min; at most 9           */
    double g[3];             /* uniform body-force density                                */
    double kolmogorov_amp;   /* adds F_x = amp * sin(2 pi y / ny); 0 = off                */
    double wall_u;           /* sliding y-walls (needs wall_y): the wall at y = ny-1/2
                                moves with velocity (+wall_u, 0, 0), the one at y = -1/2
                                with (-wall_u, 0, 0): shear 2 wall_u / ny, as for the
                                confined bijel of Sec. "High-performance LB code for
                                bijel materials". A link that comes back from a moving
                                wall gains 6 w_i rho c_i.u_w (moving-wall halfway
                                bounce-back, rho the node's density). |wall_u| < 0.3.  */
    double rho0;             /* reference density of the FP16/BF16 deviation storage and of
                                the FP16 reduced form's totals (1)                        */
    int model;               /* lbm_model: LBM_MODEL_COLOUR (default) or LBM_MODEL_SHAN_CHEN */
    double G_sc;             /* Shan-Chen coupling G_C, > 0 repulsive (Shan-Chen model)    */
    int storage;             /* lbm_storage                                               */
    void* cuda_stream;       /* cudaStream_t to run on, or NULL                           */
    int inplace;             /* 1 = one population copy, updated in place (AA pattern):
                                even steps leave a node's post-collision populations at
                                the node with opposite directions, odd steps at the
                                downstream neighbours; two passes per step (colour field,
                                then stream-collide-push), 2/3 of the two-copy memory.
                                Colour model, storage FP32/FP16/BF16, no sliding walls;
                                lbm_get_planes/lbm_set_planes and the engine refuse it.
                                0 = two copies (default).                                */
} lbm_params;

/* Number of directions and the velocity set used by lbm_get_pops/lbm_set_pops:
 * c[i] for i = 0..18, lexicographic in (c_z, c_y, c_x); the opposite of i is 18-i
 * and the rest velocity is i = 9. Writes 57 ints (c_x, c_y, c_z per direction).  */
#define LBM_Q 19
void lbm_velocity_set(int c[LBM_Q * 3]);

/* Allocates a context and all its device memory (two population copies, two
 * colour-field buffers). Returns LBM_EINVAL for nx/ny/nz < 1, tau <= 1/2,
 * beta outside [0,1], negative A_nc or h_min, unknown storage. *out is set to
 * NULL on failure.                                                              */
lbm_status lbm_create(const lbm_params* p, lbm_ctx** out);

/* Initial state: f_i^k = f_i^eq(rho_k, u) of Eq. (2) per species, with u the
 * common velocity ([3][N], NULL = 0); both colour-field buffers are set to
 * (rho_r - rho_b)/(rho_r + rho_b). rho_r + rho_b must be > 0 at every node.
 * Resets the step counter. on_device = 0: host arrays; pinned host memory mapped
 * into the device's address space (cudaHostAlloc) is read by the kernel directly,
 * other host memory is copied through a device staging buffer first (allocated on
 * first use, 7 doubles per node). Returns after the host arrays have been read.  */
lbm_status lbm_set_fields(lbm_ctx* ctx, const double* rho_r, const double* rho_b,
                          const double* u, int on_device);

/* Pinning sites ([N] bytes, nonzero = pin; NULL clears): a pin acts as another
 * interface on the nodes whose previous-step colour gradient is >= 1e-3 and that
 * lie within the cube of half-width ceil(h_cut) <= 9 around it, adding A_h[d] to
 * their near-contact strength (d = distance to the nearest pin).               */
lbm_status lbm_set_pin_mask(lbm_ctx* ctx, const uint8_t* mask, int on_device);

/* Advances n >= 0 time steps (asynchronous on the context stream). With A_nc > 0
 * each step first measures the near-contact strength A_h[h] of every node on the
 * colour field of the previous step (film thickness h along minus its gradient,
 * lag 1), then runs the fused step, where F_rep = A_h G with the current G.     */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* As lbm_step, but synchronising after every step and timing its kernels with CUDA
 * events on the context stream, summed over the n steps: out_ms[0] the near-contact
 * pass (0 when A_nc == 0; it includes the ghost-copy fill of the step's input),
 * out_ms[1] the fused step kernel, out_ms[2] the ghost-copy fill of the periodic
 * axes (0 when A_nc > 0). For measurement; it serialises the host with the device. */
lbm_status lbm_step_timed(lbm_ctx* ctx, int n, double out_ms[3]);

/* Kernel launches one lbm_step makes per time step: the fused step, and either the
 * ghost-copy fill of the periodic axes (A_nc == 0) or the near-contact pass, which
 * writes those ghost copies too (A_nc > 0). In place (inplace = 1): the colour-field
 * and collide passes, and the near-contact pass when A_nc > 0.                   */
int lbm_launches_per_step(const lbm_ctx* ctx);

/* Fields of the last step (any pointer may be NULL): rho_r, rho_b, phi [N] and the
 * physical velocity u = (j + F/2)/rho of the EDM scheme, [3][N]. Before the first
 * step, the fields that were set. Synchronises the stream. on_device = 0: host
 * arrays, written by the kernel directly when they are all pinned host memory
 * mapped into the device's address space, else through the staging buffer.      */
lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho_r, double* rho_b, double* u,
                          double* phi, int on_device);

/* Near-contact strength A_h[h] (Eq. 11) of every node ([N] float64), measured on
 * the current colour field -- the field the next step's film measurement reads --
 * exactly as that step will measure it; 0 where no film is within h_cut or
 * A_nc == 0. For diagnostics and tests; synchronises the stream.                 */
lbm_status lbm_get_nc_field(lbm_ctx* ctx, double* ah, int on_device);

/* Droplet census of the current colour field (the dense-emulsion workload reports
 * the number of droplets and their sizes): the connected components of {phi > 0}
 * under 26-connectivity (face, edge and corner neighbours), wrapping around periodic
 * axes and not across walls. *count = number of components; sizes[0 .. min(count,
 * capacity) - 1] = their node counts in descending order (sizes may be NULL when
 * capacity is 0). Diagnostic, not part of the time step; needs 8 bytes per node of
 * staging and at most 2^31 - 1 nodes. Synchronises the stream.                   */
lbm_status lbm_droplets(lbm_ctx* ctx, long long* count, long long* sizes, long long capacity);

/* Radially averaged structure factor of the current colour field (the gel workload
 * reports its peak): S(k_b) = sum over modes in shell b of |phi_hat(m)|^2 /
 * (N * modes in shell b), phi_hat the discrete Fourier transform of phi - mean(phi),
 * k(m) = 2 pi (m_x/n_x, m_y/n_y, m_z/n_z), shell b = round(|k| / dk),
 * dk = 2 pi / max(n_x, n_y, n_z), b = 0 .. nbins - 1 (modes beyond are dropped). Writes
 * S[nbins], and when not NULL k[nbins] = b dk and modes[nbins]. Every axis is treated
 * as periodic. Single-precision FFT (cuFFT) with FP64 shell sums. Synchronises.  */
lbm_status lbm_structure_factor(lbm_ctx* ctx, int nbins, double* k, double* S,
                                long long* modes);

/* Self-test of failure detection without a GPU fault: runs a kernel whose bounded
 * mbarrier wait (the kind the step kernel uses for its staged copies) can never
 * complete, so it gives up after a short bound and sets the context's error word.
 * Returns LBM_ETIMEOUT when that happened as designed, then clears the word: the
 * context stays usable. (No counterpart in the paper.) Synchronises.            */
lbm_status lbm_selftest_timeout(lbm_ctx* ctx);


/* Raw populations as float64 [19][N] per species, in the order of
 * lbm_velocity_set, plus the colour field of the previous step (lag buffer, [N];
 * may be NULL). get synchronises; set replaces the state (step counter kept).   */
lbm_status lbm_get_pops(lbm_ctx* ctx, double* f_r, double* f_b, double* phi_lag,
                        int on_device);
lbm_status lbm_set_pops(lbm_ctx* ctx, const double* f_r, const double* f_b,
                        const double* phi_lag, int on_device);

/* The same data for the sub-box of wx x wy x wz nodes starting at node (x0, y0, z0):
 * f_r, f_b float64 [19][wz][wy][wx], phi_lag [wz][wy][wx] (may be NULL), wrapped
 * around periodic axes. 1 <= w <= n per axis; along a walled axis the box must lie
 * inside the lattice. Lets a caller inspect (or check against a reference) part of
 * a lattice too large to copy out whole. Allocates a temporary device buffer of
 * 39 wx wy wz doubles; synchronises the stream.                                  */
lbm_status lbm_get_window(lbm_ctx* ctx, int x0, int y0, int z0, int wx, int wy, int wz,
                          double* f_r, double* f_b, double* phi_lag, int on_device);

/* Z-slab domain decomposition (the paper's MPI domain decomposition of the fluid, Sec.
 * "High-performance LB code for bijel materials"): the stored state of a range of z
 * planes, copied as stored, so that neighbouring subdomains can exchange halo planes
 * bitwise in every storage format. The state of plane z is every stored population
 * block's plane z (ghost cells included) and plane z of the lagged colour field (the
 * field the next step's near-contact pass reads).
 * lbm_planes_bytes: bytes of h planes of that state (the buffer of the two calls below),
 * laid out [stored blocks][h][padded plane] elements, then [h][ny][nx] float32.
 * lbm_get_planes / lbm_set_planes: planes z0 .. z0+h-1 (0 <= z0, z0 + h <= nz, h >= 1)
 * into / from `buf`, CUDA device memory the caller owns on the context's device.
 * Queued on the context's stream, no allocation, no synchronisation. Setting planes
 * replaces that part of the state; the near-contact pass needs no other state (it
 * measures every node's film anew each step).                                     */
size_t lbm_planes_bytes(const lbm_ctx* ctx, int h);
lbm_status lbm_get_planes(lbm_ctx* ctx, int z0, int h, void* buf);
lbm_status lbm_set_planes(lbm_ctx* ctx, int z0, int h, const void* buf);

/* FP64 conserved totals of the current state, summed on the device in a fixed
 * order: out = {sum f^r, sum f^b, P_x, P_y, P_z, steps, 0, 0}, P = sum_i c_i f_i.
 * Synchronises the stream.                                                      */
lbm_status lbm_observables(lbm_ctx* ctx, double out[8]);

/* Laplace-law measurement of a static droplet centred at c (FP64 on the device):
 * V = sum (1+phi)/2, R_eff = (3V/4pi)^(1/3), p = rho/3, p_in = mean p over
 * r < R_eff-3, p_out = mean p over r > R_eff+5 (minimum image on periodic axes).
 * out = {p_in - p_out, R_eff, p_in, p_out, V}. Synchronises the stream.         */
lbm_status lbm_laplace(lbm_ctx* ctx, const double centre[3], double out[5]);

/* Checkpoint: lbm_state_bytes() bytes hold the populations in their storage
 * format, both colour-field buffers and the step counter. Restoring into a
 * context with the same parameters continues bitwise identically.              */
size_t lbm_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_save_state(lbm_ctx* ctx, void* host_buf);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* host_buf);

/* Conserved totals of a population array the caller owns, computed without
 * allocating any memory -- for callers that cannot call cudaMalloc (code running
 * while a CUDA graph is being captured, processes whose device memory is handed out
 * by their own pool allocator, or latency-critical loops where an allocation's
 * implicit synchronisation is not acceptable). The paper has no counterpart; it is
 * a variant of the reduction behind lbm_observables.
 *   pops    device pointer, float32 populations [2 species][19 directions][n_nodes]
 *           in the order of lbm_velocity_set (node order is irrelevant: it is a sum)
 *   n_nodes number of nodes, 1 <= n_nodes <= 134217728 (512^3): larger arrays are
 *           rejected with LBM_EINVAL, because the partial sums live in a fixed
 *           1 MiB device array of the library (16384 blocks of 8192 nodes)
 *   out     device pointer to 5 doubles: {sum f^r, sum f^b, P_x, P_y, P_z}
 *   cuda_stream  cudaStream_t to run on, or NULL; the call is asynchronous.
 * No cudaMalloc, cudaFree or allocating library routine is called. The first call
 * on a device looks up the device address of the scratch array (make that first
 * call before any stream capture). All calls share the scratch array: calls that
 * may overlap on the GPU (different streams) race and give wrong results. Every
 * call overwrites the partial sums it reads, so nothing has to be cleared between
 * calls. Errors: LBM_EINVAL (null pointer, size), LBM_ECUDA; message in
 * lbm_last_error(NULL).                                                         */
lbm_status lbm_totals_noalloc(const float* pops, long long n_nodes, double* out,
                              void* cuda_stream);

/* Blocks until the context's queued work is done.                               */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Bytes of device memory held by a context with these parameters (admission).  */
size_t lbm_footprint_bytes(const lbm_params* p);

/* Work split the step kernel of a context with these parameters uses on a GPU with
 * num_sms SMs (host computation, no device needed). The kernel's CTAs own 32 x 8
 * tiles of (x, y) columns and march along z, two CTAs per SM. out[0] = zparts: part
 * mode, z cut into this many equal parts, one CTA per (part, tile); out[1] = chain
 * (> 0: chain mode with this many CTAs, 0: part mode); out[2], out[3] = band_k,
 * band_h: in chain mode CTAs c < band_k tiles march tile c mod tiles over planes
 * (c / tiles) band_h ... + band_h - 1, the others share the (tile, plane) units of
 * planes band_k band_h ... nz - 1 in equal contiguous runs (column-major tile order,
 * planes ascending within a tile); out[4] = grid (CTAs launched). LBM_EINVAL for
 * invalid parameters or num_sms < 1.                                              */
lbm_status lbm_work_split(const lbm_params* p, int num_sms, long long out[5]);

/* Number of steps taken since the last lbm_set_fields.                          */
long long lbm_steps_taken(const lbm_ctx* ctx);

/* Releases the context and its device memory. NULL is a no-op.                  */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failed call on this context (or of lbm_create when ctx is
 * NULL). Valid until the next call on the same context.                          */
const char* lbm_last_error(const lbm_ctx* ctx);

/* ------------------------------------------------------------------------------
 * Serving engine: independent lattices ("requests": droplet or emulsion design runs
 * of any box size) kept resident on the device and advanced together. The paper
 * has no counterpart; it is the batching and serving layer around the step above.
 *
 * - Requests are queued by lbm_engine_submit and admitted by lbm_engine_tick, in
 *   the order of the admission policy, while the device memory of the resident
 *   lattices (their lbm_footprint_bytes plus 56 bytes of host-exchange staging per
 *   node) stays within hbm_budget_bytes and at most max_slots are resident.
 *   Admission stops at the first request in that order that does not fit. A
 *   request that can never fit is refused at submission (LBM_ENOMEM).
 * - Every tick advances all resident lattices by the same number of steps k (at most
 *   chunk_steps, and not past any lattice's last step): the lattices of one storage
 *   format and relaxation class advance in one batched launch of the step kernel
 *   (CTAs of all lattices in one grid) followed by one batched ghost fill, captured
 *   in a CUDA graph of two steps that is replayed k/2 times and re-captured when the
 *   resident set changes. Lattices that reach their last step retire at the end of
 *   the tick: their fields are copied to host memory and their device memory is
 *   released, so queued requests are admitted at the next tick (continuous
 *   batching).
 * - Block schedule: each lattice's z range is cut into parts of at most T planes
 *   (one CTA per part and 32 x 8 tile); T is chosen per batch composition by timing
 *   the candidates T = 8, 16, 32, 64, 128 on the first tick of a new composition
 *   (the timed steps are real steps of the requests) and remembered.
 * - A request's result does not depend on the other requests or on the schedule:
 *   every node is computed by the same arithmetic in any batch.
 * - Requests with A_nc > 0 are served too, but not batched: each such lattice is
 *   advanced by the same k steps through its own step path (near-contact pass, then
 *   the step kernel; as lbm_step) on the engine's stream, after the batched launches
 *   of the tick.
 * An engine is not thread-safe; its calls run on its stream and synchronise it.  */
typedef struct lbm_engine lbm_engine;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory the resident lattices may hold          */
    int max_slots;            /* resident lattices at most (>= 1)                      */
    int chunk_steps;          /* steps per tick at most (>= 2)                         */
    int autotune;             /* 1: time the block-schedule candidates; 0: T = 32      */
    int policy;               /* admission order: 0 first come first served; 1 shortest
                                 job first (fewest node-steps; ties by arrival), which
                                 lowers the mean and median latency of a saturated
                                 stream                                                */
    void* cuda_stream;        /* cudaStream_t of all engine work, or NULL              */
} lbm_engine_params;

lbm_status lbm_engine_create(const lbm_engine_params* p, lbm_engine** out);

/* Queues a request: a lattice with parameters p (p->cuda_stream is ignored) and
 * initial fields as for lbm_set_fields (host arrays, copied; u may be NULL), to be
 * advanced `steps` >= 1 steps. *ticket identifies it (> 0). Requests of either
 * model and storage format are served, with or without the near-contact force.    */
lbm_status lbm_engine_submit(lbm_engine* e, const lbm_params* p, const double* rho_r,
                             const double* rho_b, const double* u, long long steps,
                             long long* ticket);

/* Withdraws a request: a queued one leaves the queue, a resident one is freed
 * (after the engine's queued work has drained) and the others go on unchanged, a
 * finished one's result is dropped. Its state becomes 5 (cancelled). LBM_ESTATE if
 * its result was taken or it failed or was cancelled already.                  */
lbm_status lbm_engine_cancel(lbm_engine* e, long long ticket);

/* One round: admit, advance, retire (see above). Writes (any pointer may be NULL)
 * the number of resident lattices after admission, of queued requests left, of
 * requests retired by this tick, and of steps k advanced. Synchronises.          */
lbm_status lbm_engine_tick(lbm_engine* e, int* resident, int* queued, int* retired,
                           int* steps_advanced);

/* State of a request: 0 queued, 1 resident, 2 finished (result ready), 3 result
 * taken, 4 failed, 5 cancelled, -1 unknown ticket.                               */
int lbm_engine_state(const lbm_engine* e, long long ticket);

/* Fields of a finished request (host arrays, any may be NULL; layouts as for
 * lbm_get_fields) and info = {steps done, tick of submission, tick of admission,
 * tick of retirement}. The result is released afterwards (state 3). LBM_ESTATE if
 * the request has not finished.                                                 */
lbm_status lbm_engine_result(lbm_engine* e, long long ticket, double* rho_r, double* rho_b,
                             double* u, double* phi, long long info[4]);

/* Engine counters: {ticks, resident, queued, device bytes held, peak device bytes,
 * block-schedule T in use, batched launches per step}.                          */
void lbm_engine_stats(const lbm_engine* e, long long out[7]);

/* Releases the engine, its resident lattices and unreturned results. NULL: no-op. */
void lbm_engine_destroy(lbm_engine* e);

/* Message of the last failed engine call.                                        */
const char* lbm_engine_last_error(const lbm_engine* e);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
