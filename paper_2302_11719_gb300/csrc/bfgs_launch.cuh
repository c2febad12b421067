// Host side of the BFGS repair that is not declared with the other launchers:
// the launch shape shared by the kernels of both state kinds and the launcher
// of the curvilinear-state kernel (curv_repair.cu).
#pragma once

#include "kernels.cuh"

namespace smppi {

// Blocks of `wpb` warps (one sequence per warp at a time) for a kernel whose
// dynamic shared memory is fixed_bytes + wpb * warp_bytes: wpb as large as fits
// (at most 4), as many blocks as are resident on `sms` SMs, no more warps than
// sequences, and few enough warp slots that their H slices (n = 2 N_r, n^2
// floats each) fit in 256 MB.  Returns the block count (0: no fit).
int bfgs_shape(const void* kern, size_t fixed_bytes, size_t warp_bytes, int N_r, int n_seq,
               int sms, int* wpb_out);

// Launch shape of the curvilinear-state BFGS repair (as bfgs_grid).
int curv_bfgs_grid(const DevParams& P, int n_seq, int sms, int* wpb_out);

// BFGS repair on the curvilinear state (smppi_repair mode 2 with state_kind 1):
// as launch_repair_bfgs, with the curvature samples `kappa` (n_track + 1
// floats) in place of the segment records; the tape keeps every state.
cudaError_t launch_repair_bfgs_curv(const DevParams& P, const float* kappa, int n_seq,
                                    const float* x0, const float* V_in, float* V_out, int n_iters,
                                    void* ws, int grid, int wpb, double* merit_out, int* iters_out,
                                    const ApplyArgs& ap, unsigned* status, cudaStream_t st);

}  // namespace smppi
