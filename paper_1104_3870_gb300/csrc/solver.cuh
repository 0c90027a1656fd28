// Solver entry points shared between solver.cu (even-odd BiCGStab with FP64
// defect correction) and precond.cu (flexible GCR with the learned preconditioner).
#pragma once
#include "dirac.cuh"

namespace laph {

// Solves K x = b for right-hand sides [first, first+nr) of the ABI arrays with the even-odd
// BiCGStab path of prm.mode (PLAIN_FP64 or MIXED_FP32); writes sol and rep[first..].
void solve_block(laph_ctx *ctx, const DiracOp &op, const c64 *rhs, c64 *sol, int first, int nr,
                 const laph_solver_params &prm, laph_solve_report *rep, cudaStream_t s);

// Same contract with FP64 defect correction around FP32 flexible GCR preconditioned by the
// network of weights (device pointer, layout of laph_precond_train).
void solve_block_learned(laph_ctx *ctx, const DiracOp &op, const float *weights, const c64 *rhs, c64 *sol, int first,
                         int nr, const laph_solver_params &prm, laph_solve_report *rep, cudaStream_t s);

}  // namespace laph
