// mrrr_launch.h -- host-side launchers of the solver's kernels (one per
// stage), implemented next to the kernels in each .cu file.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mrrr_internal.cuh"

namespace mrrr {

struct ProblemArgs {
  int batch;
  const int64_t* d_off;  // nullptr: a single problem given by the scalars below
  const int* il;
  const int* iu;
  const int64_t* w_off;
  const int64_t* z_off;
  int n;                 // single-problem scalars
  int il1, iu1;          //   range computed
  int64_t ldz;
  int slice;             //   a slice call: returns ol1..ou1 of the computed range
  int ol1, ou1;
};

// The solver's stages, in launch order (names of the per-stage profile).
enum StageId : int {
  ST_PREP = 0, ST_ROOT, ST_BISECT_ROOT, ST_RANK, ST_CLASSIFY, ST_PREREFINE, ST_CHILDREP, ST_REFINE, ST_FINAL,
  ST_VECTORS, ST_COUNT
};
extern const char* const kStageNames[ST_COUNT];
int stage_index(const char* name);  // -1 for names outside the table ("start")

// Per-stage timing and launch counting of a solve, summed by stage name.
// Direct launches: CUDA events recorded between stages, from a pool created
// once per plan (no event is created inside a timed solve).  Inside a CUDA
// graph, where a level body runs once per loop iteration: a one-thread kernel
// per stage boundary adds the GPU global timer's advance to the stage's
// counter in the workspace (Ctl::stage_ns), read back by the profile call.
struct StageTimer {
  bool on = false;
  bool device = false;       // device-clock marks (graph capture)
  Ctl* dev_ctl = nullptr;    // their accumulators
  int count = 0;
  int64_t launches = 0;
  cudaEvent_t ev[256];
  bool ev_ready = false;
  const char* name[256];
  // results of the last solve
  int nstages = 0;
  const char* stage_name[32];
  double stage_ms[32];
  void begin(cudaStream_t s);
  void mark(const char* what, cudaStream_t s);
  void finish();
  void release();
};
// The timer of the solve running on this host thread (set by the solve).
StageTimer* stage_timer();
void set_stage_timer(StageTimer* t);
inline void mark_stage(const char* what, cudaStream_t s) {
  StageTimer* t = stage_timer();
  if (t) t->mark(what, s);
}
// count one kernel launch of the current solve
inline void count_launch(int k = 1) {
  StageTimer* t = stage_timer();
  if (t) t->launches += k;
}

struct Grid {
  int nsm;
  int slot_blocks;  // grid of the per-slot kernels
  int vec_blocks;   // grid of the eigenvector kernel
  int tpb;          // threads per block of the interval kernels
};

// setup: problem table, norms and splitting, blocks, root representations,
// root bisection, output ranks of split problems
void launch_setup(const Dev& v, const ProblemArgs& a, int64_t n_total, const Grid& g, cudaStream_t s);

// one cluster level: classification and, when clusters appeared, child
// representations and refinement (second half launched by launch_level_children)
// (cond, use_cond: the condition of a CUDA graph's while node that runs one
// level per iteration)
void launch_level_classify(const Dev& v, const Grid& g, cudaStream_t s, cudaGraphConditionalHandle cond = 0,
                           int use_cond = 0);
void launch_level_children(const Dev& v, const Grid& g, cudaStream_t s);

// interval engine: mode 0 root bisection, 1 cluster pre-refinement in the
// parent, 2 refinement in the child, 3 singletons to full accuracy (see
// mrrr_engine.cu); n_total sizes the FP32 root copy of mode 0
void launch_engine(const Dev& v, int mode, const Grid& g, cudaStream_t s, int64_t n_total = 0);

// eigenvectors (one twisted factorization each), the orthogonality safeguard,
// normalisation and ordering of split problems
void launch_vectors(const Dev& v, const Grid& g, cudaStream_t s);

}  // namespace mrrr
