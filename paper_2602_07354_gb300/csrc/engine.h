// Host-side engine shared by single solves, batches and the solve server: a table of problems
// (one RVE grid with one load case each), the work-item maps of the persistent kernels, the
// recorded CUDA graph of a batch of PCG iterations, and the solve loop of Algorithm 2.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "elas_internal.h"

namespace elas {

struct Engine {
  bool mixed = false;
  int sm_count = 0;
  cudaStream_t stream = nullptr;      // owner's stream: all work is ordered on it
  cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
  std::vector<Prob> probs;            // host mirror of the device descriptors
  long long n_apply = 0, n_vec = 0;   // work items of the operator and vector kernels
  long long* d_counts = nullptr;
  Prob* d_probs = nullptr;
  int* d_item = nullptr;
  int* d_vitem = nullptr;
  SolveSetup* d_setups = nullptr;
  int* d_idx = nullptr;               // problem indices of a partial set-up (server admissions)
  DevState* d_states = nullptr;       // one solver state per problem (contiguous)
  DevState* h_states = nullptr;       // pinned host mirror of the problems' states
  int cap_probs = 0;                  // capacity of the tables (problems)
  long long cap_apply = 0, cap_vec = 0;
  BatchDev bd{};
  cudaGraphExec_t exec = nullptr;
  int exec_k = 0;
  size_t fixed_smem32 = 0, fixed_smem64 = 0, fixed_smemff = 0;  // non-zero: fixed launch shape (server)
};

// Record (or reuse) the CUDA graph of K PCG iterations over the engine's problems.
int record_batch(Engine& e, int K, std::string* err);

// Bytes of device tables for an engine with these capacities (carved from the owner's workspace).
size_t engine_table_bytes(int cap_probs, long long cap_apply, long long cap_vec);

// Item counts of one grid under its tiling.
inline long long tiles_of(const Tiling& t) { return t.n_tiles; }
inline long long chunks_of(long long N) { return (N + kVecChunk - 1) / kVecChunk; }

// Prepare an engine: tables in `mem` (engine_table_bytes), streams and pinned state mirror.
int engine_init(Engine& e, bool mixed, int sm_count, int apply_threads, int cap_probs, long long cap_apply,
                long long cap_vec, char* mem, cudaStream_t stream, std::string* err);
// Install the problem descriptors (geometry, tiling, pointers filled by the caller; the state
// pointer is assigned here from the engine's table): computes the item offsets and maps, the
// launch configuration, and uploads the tables.
int engine_set_problems(Engine& e, const std::vector<Prob>& probs, std::string* err);
// Re-upload descriptors after pointer changes (same geometry and tiling).
int engine_upload_probs(Engine& e, std::string* err);
// Algorithm 2 for every problem: state setup, initial residual, batches of K iterations until
// every problem stopped, the mixed path's FP64 w, and the FP64 true residual of every w.
// setups: host, one per problem.  *launches: kernel launches enqueued.  States end in h_states.
int engine_solve(Engine& e, const std::vector<SolveSetup>& setups, int K, int* launches, std::string* err);
void engine_destroy(Engine& e);
// FP64 products in double-float arithmetic (on, the default) or in native FP64 instructions.
void engine_set_ff64(Engine& e, bool on);

// ---- per-grid host preparation (shared by contexts, batches and the server) ------------------
struct GridHost {
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  int n_phases = 0;
  std::vector<double> cglob;   // n_phases x 36 sample-frame stiffness (zero for pores)
  std::vector<double> coef64;  // n_phases x kCoefStride modal coefficients
  std::vector<float> coef32;
  std::vector<double> cfull;   // n_phases x 21 packed stiffness
  std::vector<long long> count;  // voxels per phase
};
// Validate the inputs of Sec. 2.1.3 stages 1-3 and build the per-phase tables (Eq. 4 rotation).
int grid_prepare(GridHost& g, int nx, int ny, int nz, const int32_t* phase, int n_phases, const double* C_local,
                 const double* rodrigues, std::string* err);
// Per-phase sigma = C E for a load (6 per phase) and the no-cancellation scale of b squared.
double grid_sigma(const GridHost& g, const double* e6, std::vector<double>& sig);
void strain_tensor(const double* e6, double E[9]);
// Operator tiling for a grid at a precision: an autotuned choice if one was recorded, else the
// cost model's.
Tiling choose_tiling(const Geo& geo, int elem_bytes, int sm_count);
void record_tuned_tiling(const Geo& geo, int elem_bytes, int sm_count, const Tiling& t);
// Upper bound of a grid's operator items under any tiling the library picks.
long long max_tiles_bound(long long N);
// Autotuner: time the operator product of proto's grid (precision eb bytes) under the cost
// model's tiling and its best-ranked alternatives through the one-problem engine e (proto's h ->
// Ah), record the fastest as this grid size's schedule and return it.
int tune_tiling(Engine& e, const Prob& proto, int eb, int sm_count, long long max_tiles, int max_candidates,
                Tiling* best, double* best_ms, std::string* err);

}  // namespace elas
