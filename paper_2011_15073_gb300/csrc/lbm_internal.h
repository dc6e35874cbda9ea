// lbm_internal.h -- library-private declarations shared by the CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

// Device buffers of one run.  Distribution planes: f0..f8 then g0..g4, each
// `plane` elements apart, rows `pitch` elements apart (pitch a multiple of 64
// elements so that rows start 128-byte aligned for every storage type).
struct Buffers {
    void *dist[2] = {nullptr, nullptr};  // 14 planes in the storage type
    void *tau[2] = {nullptr, nullptr};   // 1 plane (double for F64, else float)
};

// The storages rounded stochastically (their step kernels draw random bits
// from a per-step seed).
constexpr bool rounds_stochastically(int prec) { return prec == LBM_F16S || prec == LBM_BF16S; }

struct Launch {
    const void *src;
    void *dst;
    const void *tsrc;
    void *tdst;
};

}  // namespace lbm

struct lbm_ctx {
    int nx = 0, ny = 0;
    int device = 0;
    lbm_opts opts{};
    lbm_lattice lat{};
    int64_t pitch = 0, plane = 0;  // elements
    size_t dist_elem = 0, tau_elem = 0;
    lbm::Buffers buf;
    int cur = 0;  // buffer holding the current post-collision state
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *d_small = nullptr;   // 16 doubles of small device results
    double *h_small = nullptr;   // pinned mirror of d_small
    double *d_stage = nullptr;   // lazily allocated FP64 staging (15 planes)
    double *d_snap = nullptr;    // residual snapshot u_x, u_y, T [3][ny][nx]
    double *d_part = nullptr;    // per-block partial sums of the residual
    int n_part = 0;
    double *d_nuloc = nullptr;   // local hot-wall Nu [ny]
    void *d_da = nullptr;        // per-node Darcy numbers (compute type), or null
    // Replayed step graphs (lbm_step), one per parity of the buffer state
    // (two-buffer: which buffer is current; in place: odd-step form).
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
    int graph_len = 0;
    // Stochastic-rounding storages in step graphs: the step count a replay
    // starts at (device), and while capturing, the place of the launch being
    // captured (-1 otherwise).
    long long *d_step_base = nullptr;
    int capture_s = -1;
    bool have_snap = false;
    bool aa_form_o = false;      // in-place layout: state in the odd-step form
    int64_t steps = 0;
    // Row slab of a larger cavity (lbm_init_slab): local rows [row_lo,
    // row_hi) are the global rows [y0, y0 + row_hi - row_lo) of a cavity of
    // ny_glob rows; the local rows outside (at most one below, one above) are
    // ghost rows that lbm_halo_unpack fills with the neighbours' populations.
    // A whole cavity has row_lo = 0, row_hi = ny, y0 = 0, ny_glob = ny.
    int row_lo = 0, row_hi = 0, y0 = 0, ny_glob = 0;
};

namespace lbm {

// Host launchers (lbm_kernels.cu).  All enqueue on ctx->stream and return a
// cudaError_t from cudaGetLastError().
cudaError_t launch_init(lbm_ctx *c);
cudaError_t launch_step(lbm_ctx *c);
// Write the context's step count to d_step_base (before a step-graph replay).
cudaError_t launch_set_step_base(lbm_ctx *c);
// One step of the two-buffer layout between explicit state buffers (same
// plane geometry as the context's own).
cudaError_t launch_step_buffers(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst);
cudaError_t launch_fields(lbm_ctx *c, double *d_out5);
cudaError_t launch_nusselt(lbm_ctx *c);  // -> d_small[0..1], d_nuloc
cudaError_t launch_residual(lbm_ctx *c, bool first);  // -> d_small[2..5]
cudaError_t launch_import_f64(lbm_ctx *c, const double *d_src15, int mask);
cudaError_t launch_export_f64(lbm_ctx *c, double *d_dst15);
// In-place (AA) layout (lbm_aa.cu): one step, and the conversion of the
// odd-step form back to the canonical one (no-op if already canonical).
cudaError_t launch_aa_step(lbm_ctx *c);
cudaError_t launch_aa_normalize(lbm_ctx *c);
// Halo exchange of a row slab (lbm_kernels.cu): copy the populations that
// leave through the cut rows into d_lo / d_hi (4 planes x nx values each, in
// the storage type), and the received ones into the ghost rows.  A null
// buffer skips that side.
cudaError_t launch_halo_pack(lbm_ctx *c, void *d_lo, void *d_hi);
cudaError_t launch_halo_unpack(lbm_ctx *c, const void *d_lo, const void *d_hi);
int residual_blocks(const lbm_ctx *c);

}  // namespace lbm
