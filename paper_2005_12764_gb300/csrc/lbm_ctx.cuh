// lbm_ctx.cuh -- the library's context object and the internal entry points shared
// by the C-ABI (lbm_api.cu) and the serving engine (lbm_engine.cu). Not installed:
// callers see only the opaque lbm_ctx of include/lbm.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {
// kernels (lbm_step.cu)
cudaError_t launch_step(const StepParams& p, const CUtensorMap& map, const CUtensorMap& omap,
                        int storage, int grid,
                        cudaStream_t s);
cudaError_t launch_nc_block(const StepParams& p, const CUtensorMap& lag_map, bool tma_ok,
                            int storage, int num_sms, cudaStream_t s);
void nc_cube_box(double h_cut, int box[3]);
cudaError_t launch_nc_batched(const NcBatchLattice* tab, int nlat, long long nblocks,
                              long long ghost_total, int storage, double h_cut, int num_sms,
                              cudaStream_t s);
int nc_halo(double h_cut);
cudaError_t prepare_nc_batched(int storage, double h_cut);
long long nc_block_count(const StepParams& p);
int nc_segment_blocks(int nx, int ny, int nz, int num_sms);
cudaError_t launch_wait_selftest(int* err, cudaStream_t s);
cudaError_t launch_aa_step(const StepParams& p, int layout, int storage, int num_sms,
                           cudaStream_t s);
cudaError_t launch_ghost_fill(void* f, const StepParams& p, int storage, int num_sms,
                              cudaStream_t s);
int step_tile_x();
int step_tile_y();
int step_box_rows();
int step_box_width(int storage);
int step_ctas_per_sm();
int step_pad_x(int storage);
cudaError_t launch_step_batched(const BatchLattice* tab, int nlat, int ctas, int storage,
                                bool unit_omega, int model, cudaStream_t s);
cudaError_t launch_ghost_batched(const BatchLattice* tab, int nlat, long long cells, int storage,
                                 int num_sms, cudaStream_t s);
long long ghost_cells(const StepParams& p);
}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
    lbm_params p{};
    size_t N = 0;
    size_t elem = 4;            // bytes per stored population
    int pitch = 0, nyp = 0;     // padded row length and rows per plane (ghosts included)
    int padx = 0;               // interior offset within a padded row
    size_t P = 0;               // elements per padded [z][y][x] block
    CUtensorMap tmap[2];        // TMA load descriptors of the two population copies
    CUtensorMap smap[2];        // TMA store descriptors (interior only: x < nx, y < ny)
    CUtensorMap phimap[2];      // TMA load descriptors of the two colour fields (near-contact
                                // cubes), valid when phimap_ok
    bool phimap_ok = false;
    void* f[2] = {nullptr, nullptr};
    float* phi[2] = {nullptr, nullptr};
    float* fx_row = nullptr;
    uint8_t* pin_d2 = nullptr;
    uint8_t* pin_mask = nullptr;
    float* ah = nullptr;        // near-contact strength per node (A_nc > 0)
    double* stage = nullptr;    // device FP64 staging, grown on demand
    size_t stage_cap = 0;       // its size in doubles
    double* red = nullptr;      // reduction partials
    double* red_host = nullptr; // pinned host copy of reduction results
    int red_blocks = 0;
    int cur = 0;                // population copy holding the current state
    bool aa = false;            // in-place storage: one copy, f[0]
    int layout = 0;             // its state layout (see aa_slot)
    int pc = 0;                 // phi buffer of the last step (the other one = its lag)
    long long steps = 0;
    bool fields_set = false;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int grid = 1;               // CTAs of the step kernel (one per SM at most)
    int* err_word = nullptr;    // device error word (bounded waits)
    StepParams sp{};
    std::string err;
};

namespace lbm {
// internal helpers of lbm_api.cu used by the engine
// Parameters, tensor maps and output array of the step `ahead` steps after the
// context's next one (0 or 1; the state alternates between two buffers), for a
// lattice without near-contact force, with its z range cut into `zparts` parts.
void step_params_ahead(const lbm_ctx* c, int ahead, int zparts, BatchLattice* out);
// The same for the near-contact pass of that step (parameters with the ghost copies of
// the step's input, tensor map of the lagged colour field).
void nc_params_ahead(const lbm_ctx* c, int ahead, NcBatchLattice* out);
double ctx_h_cut(const lbm_ctx* c);
// Record that `k` steps were run on the context's buffers outside lbm_step.
void advance_state(lbm_ctx* c, long long k);
// LBM_ETIMEOUT if a bounded wait in a step kernel gave up (synchronises).
lbm_status check_errors(lbm_ctx* c);
// Number of SMs of the context's device and its stream.
int ctx_num_sms(const lbm_ctx* c);
cudaStream_t ctx_stream(const lbm_ctx* c);
void set_global_error(const std::string& msg);
// Device FP64 staging of at least `doubles` values (c->stage; grown on demand, old
// contents not kept), and recording a failure in the context's error message.
lbm_status ctx_stage(lbm_ctx* c, size_t doubles);
lbm_status ctx_fail(lbm_ctx* c, lbm_status s, const std::string& msg);
}  // namespace lbm
