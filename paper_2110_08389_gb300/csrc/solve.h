// solve.h -- the solve state machine shared by mg_solve (api.cu) and
// mg_batch_solve (batch.cu).
#pragma once
#include <cmath>

#include "mg_internal.h"

namespace tmg {

// One solve (Sec. 4: cycles until the relative residual is below tol) as a
// resumable state machine: enqueue() puts the device work up to the next norm
// read on the stream (ending with the copy of the norm to pinned host memory),
// consume() reads that norm once the stream has drained and decides the next
// step.  A solve alternates the two; a batch interleaves many problems with
// one host synchronisation per step for all of them.
struct SolveState {
  Grid *g;
  double *u;
  const double *f;
  mg_params p;
  mg_info *info;
  cudaStream_t s;
  int phase = 0;  // 0: scale norm, 1: initial residual, 2: iterating
  bool done = false;
  mg_status st = MG_OK;
  double fn = 0.0, rel = 0.0, rel0 = 0.0, prev = 0.0;  // prev: rel before the last step
  int cycles = 0, outer = 0;
  bool alt = false;  // FP32+refine, 2D: the iterate lives in Grid::u2, not in u
  // the scale norm ||f - B g|| also served as the first residual (a zeroed
  // guess: f - B g is its defect); its FP32 copy is already in r32
  bool merged = false;
};

// The early stop (mg_params.early_stop): from the third step on, true when
// the last step did not reduce the relative residual (rel / prev >= 1) or
// when, kept at that rate for the `left` steps the caps allow, it would stay
// above tol.
inline bool hopeless(int steps, double rel, double prev, int left, double tol) {
  if (steps < 3 || !(prev > 0.0)) return false;
  const double rate = rel / prev;
  return rate >= 1.0 || rel * std::pow(rate, (double)left) > tol;
}

// Steps the caps still allow after `cycles` cycles and `outer` refinement
// steps.  FP64: one cycle per step, max_cycles - cycles.  FP32+refine: every
// step runs all inner_cycles and the caps are checked after it, so a step
// still starts while cycles < max_cycles (the last one may end past
// max_cycles): ceil((max_cycles - cycles) / inner_cycles), and at most
// max_outer - outer.
inline int steps_left(bool f64, int max_cycles, int max_outer, int inner_cycles, int cycles, int outer) {
  const int c = max_cycles - cycles;
  if (f64) return c > 0 ? c : 0;
  const int by_cycles = c > 0 ? (c + inner_cycles - 1) / inner_cycles : 0;
  const int by_outer = max_outer - outer > 0 ? max_outer - outer : 0;
  return by_cycles < by_outer ? by_cycles : by_outer;
}

mg_status check_params(const Grid *g, const mg_params *p);
mg_status enqueue(SolveState &q);
// the norm the step computed: its grid's pinned copy (consume) or any value
// read back otherwise (consume_value)
void consume(SolveState &q);
void consume_value(SolveState &q, double v);
// Enqueues the copy of a finished solve's iterate from Grid::u2 back into u
// when it ended there (SolveState::alt).
mg_status finish_iterate(SolveState &q);
mg_status cuda_status(const char *where, cudaError_t e);

}  // namespace tmg

// Return early with the status of a failed call (TRY_CUDA: a CUDA runtime
// call, reported through mg_last_error).
#define TRY_CUDA(where, expr)                       \
  do {                                              \
    mg_status _st = tmg::cuda_status(where, (expr)); \
    if (_st != MG_OK) return _st;                   \
  } while (0)
#define TRY(expr)                 \
  do {                            \
    mg_status _st = (expr);       \
    if (_st != MG_OK) return _st; \
  } while (0)
