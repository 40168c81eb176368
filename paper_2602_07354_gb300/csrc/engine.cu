// Engine: problem tables, launch configuration, recorded iteration batches and the solve loop.
#include "engine.h"

#include <algorithm>
#include <cstdio>

namespace elas {

namespace {

constexpr size_t kA = 256;
size_t up(size_t x) { return (x + kA - 1) / kA * kA; }

int cfail(std::string* err, cudaError_t e, const char* what) {
  if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
  return ELAS_ERR_CUDA;
}

}  // namespace

// Record one batch of K PCG iterations (Algorithm 2 steps A-E, K times) as a CUDA graph; the
// last iteration carries the FP64 residual check / replacement between steps D and E.
int record_batch(Engine& e, int K, std::string* err) {
  if (e.exec && e.exec_k == K) return ELAS_OK;
  if (e.exec) {
    cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
  }
  cudaStream_t s = e.cap_stream;
  cudaError_t c = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (c != cudaSuccess) return cfail(err, c, "cudaStreamBeginCapture");
  cudaError_t r = cudaSuccess;
  for (int it = 0; it < K && r == cudaSuccess; ++it) {
    r = launch_apply(e.bd, e.mixed ? AK_F32_DOT : AK_F64_DOT, POST_LAMBDA, GATE_RUNNING, s);
    if (r == cudaSuccess) r = launch_pcg_update(e.bd, e.mixed, s);
    if (r == cudaSuccess && it == K - 1) {
      if (e.mixed) r = launch_w_combine(e.bd, GATE_REPLACE, s);
      if (r == cudaSuccess)
        r = launch_apply(e.bd, e.mixed ? AK_MIX_RESID : AK_F64_RESID, POST_REPLACE, GATE_REPLACE, s);
    }
    if (r == cudaSuccess) r = launch_pcg_direction(e.bd, e.mixed, s);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t c2 = cudaStreamEndCapture(s, &graph);
  if (r != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cfail(err, r, "recording the PCG batch");
  }
  if (c2 != cudaSuccess) return cfail(err, c2, "cudaStreamEndCapture");
  c = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (c != cudaSuccess) return cfail(err, c, "cudaGraphInstantiate");
  e.exec_k = K;
  return ELAS_OK;
}

size_t engine_table_bytes(int cap_probs, long long cap_apply, long long cap_vec) {
  return up(2 * sizeof(long long)) + up(sizeof(Prob) * std::max(cap_probs, 1)) + up(sizeof(int) * std::max(cap_apply, 1LL)) +
         up(sizeof(int) * std::max(cap_vec, 1LL)) + up(sizeof(SolveSetup) * std::max(cap_probs, 1)) +
         up(sizeof(int) * std::max(cap_probs, 1)) + up(sizeof(DevState) * std::max(cap_probs, 1));
}

int engine_init(Engine& e, bool mixed, int sm_count, int apply_threads, int cap_probs, long long cap_apply,
                long long cap_vec, char* mem, cudaStream_t stream, std::string* err) {
  e.mixed = mixed;
  e.sm_count = sm_count;
  e.stream = stream;
  e.cap_probs = cap_probs;
  e.cap_apply = cap_apply;
  e.cap_vec = cap_vec;
  size_t off = 0;
  e.d_counts = reinterpret_cast<long long*>(mem + off);
  off += up(2 * sizeof(long long));
  e.d_probs = reinterpret_cast<Prob*>(mem + off);
  off += up(sizeof(Prob) * std::max(cap_probs, 1));
  e.d_item = reinterpret_cast<int*>(mem + off);
  off += up(sizeof(int) * std::max(cap_apply, 1LL));
  e.d_vitem = reinterpret_cast<int*>(mem + off);
  off += up(sizeof(int) * std::max(cap_vec, 1LL));
  e.d_setups = reinterpret_cast<SolveSetup*>(mem + off);
  off += up(sizeof(SolveSetup) * std::max(cap_probs, 1));
  e.d_idx = reinterpret_cast<int*>(mem + off);
  off += up(sizeof(int) * std::max(cap_probs, 1));
  e.d_states = reinterpret_cast<DevState*>(mem + off);
  cudaError_t c = cudaMemsetAsync(e.d_states, 0, sizeof(DevState) * std::max(cap_probs, 1), stream);
  if (c != cudaSuccess) return cfail(err, c, "engine states");
  c = cudaStreamCreateWithFlags(&e.cap_stream, cudaStreamNonBlocking);
  if (c != cudaSuccess) return cfail(err, c, "engine stream");
  c = cudaMallocHost((void**)&e.h_states, sizeof(DevState) * std::max(cap_probs, 1));
  if (c != cudaSuccess) return cfail(err, c, "engine pinned state mirror");
  e.bd.probs = e.d_probs;
  e.bd.item_prob = e.d_item;
  e.bd.vitem_prob = e.d_vitem;
  e.bd.counts = e.d_counts;
  e.bd.apply_threads = apply_threads;
  e.bd.vec_threads = kVecThreads;
  e.bd.ff64 = 1;  // FP64 products in double-float arithmetic unless the owner asks for native FP64
  return ELAS_OK;
}

void engine_set_ff64(Engine& e, bool on) {
  if ((e.bd.ff64 != 0) == on) return;
  e.bd.ff64 = on ? 1 : 0;
  if (e.exec) {  // the kernel choice is part of the recorded graph
    cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
  }
}

int engine_set_problems(Engine& e, const std::vector<Prob>& probs, std::string* err) {
  if ((int)probs.size() > e.cap_probs) {
    if (err) *err = "engine: more problems than its tables hold";
    return ELAS_ERR_INVALID_ARG;
  }
  e.probs = probs;
  long long na = 0, nv = 0;
  size_t smem32 = 0, smem64 = 0, smemff = 0;
  for (size_t i = 0; i < e.probs.size(); ++i) {
    Prob& p = e.probs[i];
    p.st = e.d_states + i;
    p.item0_apply = na;
    p.item0_vec = nv;
    na += p.n_tiles;
    nv += p.n_chunks;
    smem32 = std::max(smem32, apply_smem_bytes(p.tx, p.ty, 4));
    smem64 = std::max(smem64, apply_smem_bytes(p.tx, p.ty, 8));
    smemff = std::max(smemff, apply_smem_bytes_ff(p.tx, p.ty));
  }
  if (na > e.cap_apply || nv > e.cap_vec) {
    if (err) *err = "engine: more work items than its tables hold";
    return ELAS_ERR_INVALID_ARG;
  }
  e.n_apply = na;
  e.n_vec = nv;
  std::vector<int> item(std::max(na, 1LL)), vitem(std::max(nv, 1LL));
  for (int i = 0; i < (int)e.probs.size(); ++i) {
    for (long long t = 0; t < e.probs[i].n_tiles; ++t) item[e.probs[i].item0_apply + t] = i;
    for (long long t = 0; t < e.probs[i].n_chunks; ++t) vitem[e.probs[i].item0_vec + t] = i;
  }
  const long long counts[2] = {na, nv};
  if (e.fixed_smem32) {
    // fixed launch shape: the recorded graph stays valid whatever the set of problems
    if (smem32 > e.fixed_smem32 || smem64 > e.fixed_smem64 || smemff > e.fixed_smemff) {
      if (err) *err = "engine: a problem's tile exceeds the fixed launch shape";
      return ELAS_ERR_INVALID_ARG;
    }
    e.bd.smem32 = e.fixed_smem32;
    e.bd.smem64 = e.fixed_smem64;
    e.bd.smemff = e.fixed_smemff;
    e.bd.blocks32 = e.sm_count * apply_resident_blocks(4, e.bd.apply_threads, e.bd.smem32);
    e.bd.blocks64 = e.sm_count * apply_resident_blocks(8, e.bd.apply_threads, e.bd.smem64);
    e.bd.vec_blocks = e.sm_count * 8;
    e.bd.nohalo64 = 0;  // the kernel choice is part of the recorded graph, which must outlive any set
  } else {
    e.bd.smem32 = std::max<size_t>(smem32, 16);
    e.bd.smem64 = std::max<size_t>(smem64, 16);
    e.bd.smemff = std::max<size_t>(smemff, 16);
    const int r32 = apply_resident_blocks(4, e.bd.apply_threads, e.bd.smem32);
    const int r64 = apply_resident_blocks(8, e.bd.apply_threads, e.bd.smem64);
    e.bd.blocks32 = (int)std::max(1LL, std::min<long long>(na, (long long)e.sm_count * r32));
    e.bd.blocks64 = (int)std::max(1LL, std::min<long long>(na, (long long)e.sm_count * r64));
    e.bd.vec_blocks = (int)std::max(1LL, std::min<long long>(nv, (long long)e.sm_count * 8));
    bool fits = !e.probs.empty();
    for (const Prob& p : e.probs) fits = fits && apply_nohalo_fits(p);
    e.bd.nohalo64 = fits ? 1 : 0;
  }
  cudaError_t c = cudaMemcpyAsync(e.d_counts, counts, sizeof counts, cudaMemcpyHostToDevice, e.stream);
  if (c == cudaSuccess)
    c = cudaMemcpyAsync(e.d_item, item.data(), sizeof(int) * item.size(), cudaMemcpyHostToDevice, e.stream);
  if (c == cudaSuccess)
    c = cudaMemcpyAsync(e.d_vitem, vitem.data(), sizeof(int) * vitem.size(), cudaMemcpyHostToDevice, e.stream);
  if (c != cudaSuccess) return cfail(err, c, "engine tables");
  if (e.exec && !e.fixed_smem32) {  // launch configuration may have changed: record again on next solve
    cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
  }
  return engine_upload_probs(e, err);
}

int engine_upload_probs(Engine& e, std::string* err) {
  if (e.probs.empty()) return ELAS_OK;
  cudaError_t c = cudaMemcpyAsync(e.d_probs, e.probs.data(), sizeof(Prob) * e.probs.size(), cudaMemcpyHostToDevice,
                                  e.stream);
  if (c != cudaSuccess) return cfail(err, c, "engine descriptors");
  return ELAS_OK;
}

int engine_solve(Engine& e, const std::vector<SolveSetup>& setups, int K, int* launches, std::string* err) {
  const int n = (int)e.probs.size();
  int L = 0;
  cudaStream_t s = e.stream;
  cudaError_t c = cudaMemcpyAsync(e.d_setups, setups.data(), sizeof(SolveSetup) * n, cudaMemcpyHostToDevice, s);
  if (c != cudaSuccess) return cfail(err, c, "solve setups");
  if ((c = launch_state_init(e.bd, e.d_setups, nullptr, n, s)) != cudaSuccess) return cfail(err, c, "state init");
  if ((c = launch_pcg_init(e.bd, e.mixed, s)) != cudaSuccess) return cfail(err, c, "PCG init");
  L += 2;
  int rc = record_batch(e, K, err);
  if (rc != ELAS_OK) return rc;
  int max_iter = 0;
  for (const SolveSetup& su : setups) max_iter = std::max(max_iter, su.max_iter);
  // every batch advances every running problem by at least one iteration or resolves its pending
  // residual check, so max_iter + a few batches always suffice
  const long long max_batches = (long long)max_iter + 4;
  for (long long b = 0;; ++b) {
    bool all_done = true;
    c = cudaMemcpyAsync(e.h_states, e.d_states, sizeof(DevState) * n, cudaMemcpyDeviceToHost, s);
    if (c != cudaSuccess) return cfail(err, c, "state read");
    if ((c = cudaStreamSynchronize(s)) != cudaSuccess) return cfail(err, c, "solve");
    for (int i = 0; i < n; ++i) all_done &= e.h_states[i].done != 0;
    if (all_done || b >= max_batches) break;
    if ((c = cudaGraphLaunch(e.exec, s)) != cudaSuccess) return cfail(err, c, "cudaGraphLaunch");
    L += 3 * K + 1 + (e.mixed ? 1 : 0);
  }
  if (e.mixed) {
    if ((c = launch_w_combine(e.bd, GATE_NONE, s)) != cudaSuccess) return cfail(err, c, "w combine");
    L += 1;
  }
  // FP64 true residual of every returned w
  if ((c = launch_apply(e.bd, AK_F64_NORM, POST_TRUE_NORM, GATE_NONE, s)) != cudaSuccess)
    return cfail(err, c, "true residual");
  L += 1;
  c = cudaMemcpyAsync(e.h_states, e.d_states, sizeof(DevState) * n, cudaMemcpyDeviceToHost, s);
  if (c != cudaSuccess) return cfail(err, c, "state read");
  if ((c = cudaStreamSynchronize(s)) != cudaSuccess) return cfail(err, c, "solve");
  if (launches) *launches = L;
  return ELAS_OK;
}

void engine_destroy(Engine& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.cap_stream) cudaStreamDestroy(e.cap_stream);
  if (e.h_states) cudaFreeHost(e.h_states);
  e = Engine{};
}

}  // namespace elas
