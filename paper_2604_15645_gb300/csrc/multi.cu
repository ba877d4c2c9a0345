// Many independent PINNs in one training step (pinn_multi_*).
//
// Every network keeps its own handle (its own widths, depth, point counts and
// problem).  One call of pinn_multi_train_step runs, for all of them, the whole
// step: input jets -> jet forward -> residual/loss -> adjoint -> ordered FP64
// reductions, then one fused Adam update over the concatenated parameter vector.
// The first call captures that step into a CUDA graph: the networks' launch
// sequences are forked onto worker streams (so small networks run side by side on
// the GPU), joined, and followed by the Adam launch; later calls with the same
// buffers replay the graph.  The Adam scalars that change per step (learning rate,
// step-dependent bias corrections) are written into the captured Adam node's
// arguments before each replay, so a replay needs no re-capture.
//
// pinn_multi_autotune picks, per network, the fastest kernel configuration by timing
// each: tcgen05 with the fused adjoint + weight-gradient kernel, tcgen05 with separate
// adjoint and weight-gradient kernels (weight-gradient tiles of 256 or of 128 output
// rows), or the CUDA-core GEMMs (tiles of 64 x 256), and caches the choice per (width,
// depth, point-count bucket, precision) in a JSON file.  Networks are spread over the
// worker streams longest first (each to the stream with the least estimated work so far,
// the estimate being the jet-GEMM FLOPs), so the big networks start at once and the
// small ones fill in around them.
//
// pinn_multi_set_grouped(m, 1) captures the step level by level instead: every
// network's pass runs in stages, and at each layer level the tensor-core GEMMs of all
// networks are issued as one grouped launch per kernel variant (tc.h), with the other
// launches of the level on the worker streams between a fork and a join.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "tc.h"

namespace pinn {
const void* adam_kernel();
}

struct pinn_multi {
  int n = 0;
  std::vector<pinn_handle*> nets;
  std::vector<int64_t> poff;            // parameter offsets [n + 1]
  std::vector<cudaStream_t> streams;
  cudaStream_t cap = nullptr;           // capture stream (the caller's may be the legacy default stream)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t adam_node = nullptr;
  std::string key;                      // buffers / sizes / engines the graph was captured with
  bool grouped = false;                 // tensor-core GEMMs of one level share grouped launches
  pinn::TcBatch* batch = nullptr;       // the grouped launches' collector and device table
  char err[512] = {0};
};

namespace {

constexpr int kMaxStreams = 32;

// Kernel configurations the autotuner chooses among (pinn_multi_set_config).
enum NetConfig { CFG_TC = 0, CFG_CUDA_CORES = 1, CFG_TC_UNFUSED = 2, CFG_TC_UNFUSED_DW128 = 3, CFG_COUNT = 4 };
const char* const kConfigNames[CFG_COUNT] = {"tc", "cuda_cores", "tc_unfused", "tc_unfused_dw128"};
constexpr int32_t kConfigFlags = PINN_FLAG_CUDA_CORES | PINN_FLAG_UNFUSED_ADJOINT | PINN_FLAG_DW_ROWS_128;

int32_t config_flags(int c) {
  switch (c) {
    case CFG_CUDA_CORES: return PINN_FLAG_CUDA_CORES;
    case CFG_TC_UNFUSED: return PINN_FLAG_UNFUSED_ADJOINT;
    case CFG_TC_UNFUSED_DW128: return PINN_FLAG_UNFUSED_ADJOINT | PINN_FLAG_DW_ROWS_128;
    default: return 0;
  }
}
int config_of(int32_t flags) {
  if (flags & PINN_FLAG_CUDA_CORES) return CFG_CUDA_CORES;
  if (flags & PINN_FLAG_UNFUSED_ADJOINT) return (flags & PINN_FLAG_DW_ROWS_128) ? CFG_TC_UNFUSED_DW128 : CFG_TC_UNFUSED;
  return CFG_TC;
}

// Jet-GEMM work of network i on its batch (2 MAC per jet column and weight entry).
double net_cost(const pinn_handle* h, const pinn_batch& b) {
  const double cols = 4.0 * (double)(b.n_res + b.n_ic + b.n_bc);
  double c = 0.0;
  for (int l = h->first_gemm; l < h->L; ++l) c += 6.0 * h->layers[l].fin * h->layers[l].fout * cols;
  return c;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

pinn_status set_err(pinn_multi* m, const char* msg) {
  if (m) snprintf(m->err, sizeof(m->err), "%s", msg);
  return PINN_ERR_INVALID_ARG;
}

// Workspace of network i: the larger of its two engines' needs, so switching
// engines never invalidates the caller's buffer.
pinn_status net_ws(pinn_handle* h, const pinn_batch& b, size_t* bytes) {
  const int32_t saved = h->spec.flags;
  size_t most = 0;
  pinn_status s = PINN_OK;
  for (int c = 0; c < CFG_COUNT && !s; ++c) {
    size_t x = 0;
    h->spec.flags = (saved & ~kConfigFlags) | config_flags(c);
    s = pinn_workspace_bytes(h, b.n_res, b.n_ic, b.n_bc, &x);
    most = std::max(most, x);
  }
  h->spec.flags = saved;
  *bytes = align256(most);
  return s;
}

std::string make_key(pinn_multi* m, const pinn_batch* batches, const float* p, const float* g, const float* mm,
                     const float* v, void* ws, const double* loss, void* stream) {
  std::string k;
  char buf[160];
  snprintf(buf, sizeof(buf), "%p %p %p %p %p %p %p %d|", (const void*)p, (const void*)g, (const void*)mm,
           (const void*)v, ws, (const void*)loss, stream, m->grouped ? 1 : 0);
  k += buf;
  for (int i = 0; i < m->n; ++i) {
    const pinn_batch& b = batches[i];
    snprintf(buf, sizeof(buf), "%d:%p,%lld,%p,%p,%lld,%u,%p,%p,%lld,%u,%d;", i, (const void*)b.x_res,
             (long long)b.n_res, (const void*)b.x_ic, (const void*)b.g_ic, (long long)b.n_ic, b.ic_mask,
             (const void*)b.x_bc, (const void*)b.g_bc, (long long)b.n_bc, b.bc_mask, m->nets[i]->spec.flags);
    k += buf;
  }
  return k;
}

void drop_graph(pinn_multi* m) {
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->exec = nullptr;
  m->graph = nullptr;
  m->adam_node = nullptr;
  m->key.clear();
}

// Worker stream of each network: longest processing time first, the biggest networks
// first, each to the stream with the least estimated work so far.
std::vector<int> assign_streams(const pinn_multi* m, const pinn_batch* batches) {
  const int ns = (int)m->streams.size();
  std::vector<int> order(m->n), stream_of(m->n, 0);
  std::vector<double> cost(m->n), load(ns, 0.0);
  for (int i = 0; i < m->n; ++i) { order[i] = i; cost[i] = net_cost(m->nets[i], batches[i]); }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += cost[i];
    stream_of[i] = k;
  }
  return stream_of;
}

struct AdamArgs {
  float lr, b1, b2, eps, bc1, bc2;
};

// Enqueue one whole training step on `st` (under stream capture).
pinn_status enqueue_step(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches, float* d_p, float* d_g,
                         float* d_m, float* d_v, char* ws, const std::vector<size_t>& ws_off,
                         const std::vector<size_t>& ws_sz, const AdamArgs& ad, double* d_loss, cudaStream_t st) {
  if (cudaEventRecord(m->fork, st) != cudaSuccess) return PINN_ERR_CUDA;
  const int ns = (int)m->streams.size();
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(m->streams[k], m->fork, 0) != cudaSuccess) return PINN_ERR_CUDA;
  // longest-processing-time-first: biggest networks first, each to the least loaded stream
  const std::vector<int> stream_of = assign_streams(m, batches);
  std::vector<int> order(m->n);
  std::vector<double> cost(m->n);
  for (int i = 0; i < m->n; ++i) { order[i] = i; cost[i] = net_cost(m->nets[i], batches[i]); }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int i : order) {
    pinn_status s = pinn_loss_grad(m->nets[i], &probs[i], &batches[i], d_p + m->poff[i], ws + ws_off[i], ws_sz[i],
                                   d_loss + (int64_t)i * PINN_LOSS_TERMS, d_g + m->poff[i],
                                   m->streams[stream_of[i]]);
    if (s) {
      snprintf(m->err, sizeof(m->err), "network %d: %s", i, pinn_last_error(m->nets[i]));
      return s;
    }
  }
  for (int k = 0; k < ns; ++k) {
    if (cudaEventRecord(m->joins[k], m->streams[k]) != cudaSuccess || cudaStreamWaitEvent(st, m->joins[k], 0) != cudaSuccess)
      return PINN_ERR_CUDA;
  }
  pinn::launch_adam(d_p, d_g, d_m, d_v, m->poff[m->n], ad.lr, ad.b1, ad.b2, ad.eps, ad.bc1, ad.bc2, st);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

// Table entries the grouped step can issue: one per forward GEMM, two per hidden layer
// (adjoint and weight gradient) and one to spare.
size_t grouped_entries(const pinn_multi* m) {
  size_t n = 0;
  for (const pinn_handle* h : m->nets) n += (size_t)(h->L - h->first_gemm) + 2 * (size_t)h->L + 1;
  return n;
}

// One training step with grouped tensor-core launches (under stream capture on `st`).
// Every network's pass runs in stages (internal.h), level by level over all networks:
// the per-network launches of a level (RWF weights and input jets, CUDA-core GEMMs,
// output/loss, reductions, finalisation) go to the worker streams, and the tensor-core
// GEMMs of the level are collected and issued on `st` as one grouped launch per kernel
// variant; the workers fork from `st` before a level and join it after.  The per-network
// order of the launches is that of pinn_loss_grad, and the stages of one level of one
// network touch disjoint outputs, so the results are those of the per-network step.
pinn_status enqueue_grouped(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches, float* d_p,
                            float* d_g, float* d_m, float* d_v, char* ws, const std::vector<size_t>& ws_off,
                            const std::vector<size_t>& ws_sz, const AdamArgs& ad, double* d_loss, cudaStream_t st) {
  const int n = m->n, ns = (int)m->streams.size();
  std::vector<pinn::StagedPass*> sp(n, nullptr);
  struct Cleanup {
    pinn_multi* m;
    std::vector<pinn::StagedPass*>& sp;
    ~Cleanup() {
      for (pinn::StagedPass* x : sp) pinn::staged_destroy(x);
      for (pinn_handle* h : m->nets) pinn::tc_batch_attach(h, nullptr);
    }
  } cleanup{m, sp};
  auto net_err = [&](int i, pinn_status s) {
    snprintf(m->err, sizeof(m->err), "network %d: %s", i, pinn_last_error(m->nets[i]));
    return s;
  };
  for (int i = 0; i < n; ++i) {
    pinn_status s = pinn::staged_create(m->nets[i], &probs[i], &batches[i], d_p + m->poff[i], ws + ws_off[i],
                                        ws_sz[i], d_loss + (int64_t)i * PINN_LOSS_TERMS, d_g + m->poff[i], &sp[i]);
    if (s) return net_err(i, s);
  }
  const std::vector<int> stream_of = assign_streams(m, batches);
  pinn::tc_batch_reset(m->batch);
  for (pinn_handle* h : m->nets) pinn::tc_batch_attach(h, m->batch);
  auto fork = [&]() {
    if (cudaEventRecord(m->fork, st) != cudaSuccess) return false;
    for (int k = 0; k < ns; ++k)
      if (cudaStreamWaitEvent(m->streams[k], m->fork, 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() {
    for (int k = 0; k < ns; ++k)
      if (cudaEventRecord(m->joins[k], m->streams[k]) != cudaSuccess || cudaStreamWaitEvent(st, m->joins[k], 0) != cudaSuccess)
        return false;
    return true;
  };
  // runs `stage` for every network that has it, then the level's grouped launches
  auto level = [&](auto&& stage) -> pinn_status {
    if (!fork()) return PINN_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
      const pinn_status s = stage(i, m->streams[stream_of[i]]);
      if (s) return net_err(i, s);
    }
    const pinn_status s = pinn::tc_batch_flush(m->batch, m->nets[0], st);
    if (s) return net_err(0, s);
    return join() ? PINN_OK : PINN_ERR_CUDA;
  };
  int fwd_levels = 0, bwd_levels = 0;
  for (int i = 0; i < n; ++i) {
    fwd_levels = std::max(fwd_levels, pinn::staged_forward_levels(sp[i]));
    bwd_levels = std::max(bwd_levels, m->nets[i]->L);
  }
  pinn_status s = level([&](int i, cudaStream_t ws_) { return pinn::staged_prologue(sp[i], ws_); });
  for (int l = 0; l < fwd_levels && !s; ++l)
    s = level([&](int i, cudaStream_t ws_) {
      return l < pinn::staged_forward_levels(sp[i]) ? pinn::staged_forward(sp[i], l, ws_) : PINN_OK;
    });
  if (!s) s = level([&](int i, cudaStream_t ws_) { return pinn::staged_output(sp[i], ws_); });
  for (int l = 0; l < bwd_levels && !s; ++l)
    s = level([&](int i, cudaStream_t ws_) {
      return l < m->nets[i]->L ? pinn::staged_backward(sp[i], l, ws_) : PINN_OK;
    });
  if (!s) s = level([&](int i, cudaStream_t ws_) { return pinn::staged_finalize(sp[i], ws_); });
  if (s) return s;
  pinn::launch_adam(d_p, d_g, d_m, d_v, m->poff[m->n], ad.lr, ad.b1, ad.b2, ad.eps, ad.bc1, ad.bc2, st);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

pinn_status plan_ws(pinn_multi* m, const pinn_batch* batches, std::vector<size_t>& off, std::vector<size_t>& sz,
                    size_t* total) {
  off.resize(m->n);
  sz.resize(m->n);
  size_t t = 0;
  for (int i = 0; i < m->n; ++i) {
    pinn_status s = net_ws(m->nets[i], batches[i], &sz[i]);
    if (s) return s;
    off[i] = t;
    t += sz[i];
  }
  *total = t;
  return PINN_OK;
}

}  // namespace

extern "C" {

PINN_API pinn_status pinn_multi_create(const pinn_spec* specs, int32_t n_nets, pinn_multi** out) {
  if (!specs || !out || n_nets < 1 || n_nets > 4096) return PINN_ERR_INVALID_ARG;
  *out = nullptr;
  pinn_multi* m = new (std::nothrow) pinn_multi();
  if (!m) return PINN_ERR_OOM;
  m->n = n_nets;
  m->poff.assign(n_nets + 1, 0);
  for (int i = 0; i < n_nets; ++i) {
    pinn_handle* h = nullptr;
    pinn_status s = pinn_create(&specs[i], &h);
    if (s) {
      for (pinn_handle* x : m->nets) pinn_destroy(x);
      delete m;
      return s;
    }
    m->nets.push_back(h);
    int64_t P = 0;
    pinn_param_count(h, &P);
    m->poff[i + 1] = m->poff[i] + P;
  }
  const int ns = std::min(n_nets, kMaxStreams);
  m->batch = pinn::tc_batch_create();
  bool ok = m->batch && cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; ok && k < ns; ++k) {
    cudaStream_t s;
    cudaEvent_t e;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
      m->streams.push_back(s);
      m->joins.push_back(e);
    }
  }
  if (!ok) {
    pinn_multi_destroy(m);
    return PINN_ERR_CUDA;
  }
  *out = m;
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_destroy(pinn_multi* m) {
  if (!m) return PINN_OK;
  drop_graph(m);
  for (cudaStream_t s : m->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : m->joins) cudaEventDestroy(e);
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->cap) cudaStreamDestroy(m->cap);
  pinn::tc_batch_destroy(m->batch);
  for (pinn_handle* h : m->nets) pinn_destroy(h);
  delete m;
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_param_offsets(const pinn_multi* m, int64_t* offsets) {
  if (!m || !offsets) return PINN_ERR_INVALID_ARG;
  for (int i = 0; i <= m->n; ++i) offsets[i] = m->poff[i];
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_workspace_bytes(pinn_multi* m, const pinn_batch* batches, size_t* bytes) {
  if (!m || !batches || !bytes) return PINN_ERR_INVALID_ARG;
  std::vector<size_t> off, sz;
  return plan_ws(m, batches, off, sz, bytes);
}

PINN_API pinn_status pinn_multi_set_ff_matrix(pinn_multi* m, int32_t net, const float* d_B) {
  if (!m || net < 0 || net >= m->n) return PINN_ERR_INVALID_ARG;
  drop_graph(m);
  return pinn_set_ff_matrix(m->nets[net], d_B);
}

PINN_API pinn_status pinn_multi_set_engine(pinn_multi* m, int32_t net, int32_t cuda_cores) {
  if (!m || net < 0 || net >= m->n) return PINN_ERR_INVALID_ARG;
  int32_t& f = m->nets[net]->spec.flags;
  f = (f & ~kConfigFlags) | (cuda_cores ? PINN_FLAG_CUDA_CORES : 0);
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_set_config(pinn_multi* m, int32_t net, int32_t config) {
  if (!m || net < 0 || net >= m->n || config < 0 || config >= CFG_COUNT) return PINN_ERR_INVALID_ARG;
  int32_t& f = m->nets[net]->spec.flags;
  f = (f & ~kConfigFlags) | config_flags(config);
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_get_config(const pinn_multi* m, int32_t net, int32_t* config) {
  if (!m || !config || net < 0 || net >= m->n) return PINN_ERR_INVALID_ARG;
  *config = config_of(m->nets[net]->spec.flags);
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_set_grouped(pinn_multi* m, int32_t on) {
  if (!m) return PINN_ERR_INVALID_ARG;
  m->grouped = on != 0;
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_get_grouped(const pinn_multi* m, int32_t* on) {
  if (!m || !on) return PINN_ERR_INVALID_ARG;
  *on = m->grouped ? 1 : 0;
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_get_engine(const pinn_multi* m, int32_t net, int32_t* cuda_cores) {
  if (!m || !cuda_cores || net < 0 || net >= m->n) return PINN_ERR_INVALID_ARG;
  *cuda_cores = (m->nets[net]->spec.flags & PINN_FLAG_CUDA_CORES) ? 1 : 0;
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_train_step(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches,
                                           float* d_params, float* d_grad, float* d_m, float* d_v, int64_t step,
                                           float lr, float beta1, float beta2, float eps, void* d_ws,
                                           size_t ws_bytes, double* d_loss, void* stream) {
  if (!m || !probs || !batches || !d_params || !d_grad || !d_m || !d_v || !d_ws || !d_loss || step < 1)
    return set_err(m, "NULL argument or step < 1");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
    return set_err(m, "bad Adam hyper-parameters");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256) return set_err(m, "workspace must be 256-byte aligned");
  std::vector<size_t> off, sz;
  size_t total = 0;
  pinn_status s = plan_ws(m, batches, off, sz, &total);
  if (s) return s;
  if (ws_bytes < total) {
    snprintf(m->err, sizeof(m->err), "workspace too small: %zu < %zu bytes", ws_bytes, total);
    return PINN_ERR_WORKSPACE;
  }
  char* ws = static_cast<char*>(d_ws);
  cudaStream_t st = (cudaStream_t)stream;
  AdamArgs ad;
  ad.lr = lr; ad.b1 = beta1; ad.b2 = beta2; ad.eps = eps;
  ad.bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  ad.bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  const std::string key = make_key(m, batches, d_params, d_grad, d_m, d_v, d_ws, d_loss, stream);
  if (key != m->key) {
    drop_graph(m);
    if (m->grouped) {
      // the table is rewritten below: no replay still reading it may be in flight
      if (cudaStreamSynchronize(st) != cudaSuccess || pinn::tc_batch_reserve(m->batch, grouped_entries(m)) != PINN_OK) {
        cudaGetLastError();
        snprintf(m->err, sizeof(m->err), "cannot allocate the grouped launch table");
        return PINN_ERR_OOM;
      }
    }
    // capture on the handle's own stream; the graph is launched on the caller's
    if (cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      snprintf(m->err, sizeof(m->err), "cannot begin stream capture");
      return PINN_ERR_CUDA;
    }
    s = m->grouped ? enqueue_grouped(m, probs, batches, d_params, d_grad, d_m, d_v, ws, off, sz, ad, d_loss, m->cap)
                   : enqueue_step(m, probs, batches, d_params, d_grad, d_m, d_v, ws, off, sz, ad, d_loss, m->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(m->cap, &g);
    if (s || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!s) snprintf(m->err, sizeof(m->err), "graph capture failed: %s", cudaGetErrorString(e));
      return s ? s : PINN_ERR_CUDA;
    }
    // the grouped launches' table, read by the graph's kernels from the first replay on
    if (m->grouped && pinn::tc_batch_upload(m->batch) != PINN_OK) {
      cudaGraphDestroy(g);
      snprintf(m->err, sizeof(m->err), "grouped launch table upload failed");
      return PINN_ERR_CUDA;
    }
    // find the Adam node, whose scalar arguments change from step to step
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == pinn::adam_kernel()) m->adam_node = nd;
    }
    if (!m->adam_node || cudaGraphInstantiate(&m->exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      m->exec = nullptr;
      snprintf(m->err, sizeof(m->err), "graph instantiation failed");
      return PINN_ERR_CUDA;
    }
    m->graph = g;
    m->key = key;
  } else {
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(m->adam_node, &kp) != cudaSuccess) return PINN_ERR_CUDA;
    int64_t n = m->poff[m->n];
    float* p0 = d_params;
    const float* g0 = d_grad;
    float* m0 = d_m;
    float* v0 = d_v;
    void* args[] = {&p0, &g0, &m0, &v0, &n, &ad.lr, &ad.b1, &ad.b2, &ad.eps, &ad.bc1, &ad.bc2};
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(m->exec, m->adam_node, &kp) != cudaSuccess) {
      snprintf(m->err, sizeof(m->err), "cannot update the Adam node");
      return PINN_ERR_CUDA;
    }
  }
  const cudaError_t le = cudaGraphLaunch(m->exec, st);
  if (le != cudaSuccess) {
    snprintf(m->err, sizeof(m->err), "graph launch: %s", cudaGetErrorString(le));
    return PINN_ERR_CUDA;
  }
  return PINN_OK;
}

PINN_API pinn_status pinn_multi_status_poll(pinn_multi* m, void* stream) {
  if (!m) return PINN_ERR_INVALID_ARG;
  pinn_status worst = PINN_OK;
  for (pinn_handle* h : m->nets) {
    pinn_status s = pinn_status_poll(h, stream);
    if (s && !worst) worst = s;
  }
  return worst;
}

PINN_API const char* pinn_multi_last_error(const pinn_multi* m) { return m ? m->err : "NULL handle"; }

// Autotuner: time every applicable kernel configuration per (width, depth, point
// bucket, precision) and keep the fastest.  The cache file holds one JSON object of
// "key": "tc" | "cuda_cores" | "tc_unfused" | "tc_unfused_dw128".
PINN_API pinn_status pinn_multi_autotune(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches,
                                         const float* d_params, void* d_ws, size_t ws_bytes, double* d_loss,
                                         float* d_grad, const char* cache_path, void* stream) {
  if (!m || !probs || !batches || !d_params || !d_ws || !d_loss || !d_grad) return set_err(m, "NULL argument");
  std::vector<size_t> off, sz;
  size_t total = 0;
  pinn_status s = plan_ws(m, batches, off, sz, &total);
  if (s) return s;
  if (ws_bytes < total) return PINN_ERR_WORKSPACE;
  std::map<std::string, int> cache;   // key -> configuration
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[256], k[128], v[32];
      while (fgets(line, sizeof(line), f))
        if (sscanf(line, " \"%127[^\"]\" : \"%31[^\"]\"", k, v) == 2)
          for (int c = 0; c < CFG_COUNT; ++c)
            if (strcmp(v, kConfigNames[c]) == 0) cache[k] = c;
      fclose(f);
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    snprintf(m->err, sizeof(m->err), "autotune: cannot create timing events");
    return PINN_ERR_CUDA;
  }
  drop_graph(m);
  for (int i = 0; i < m->n && !s; ++i) {
    pinn_handle* h = m->nets[i];
    const pinn_batch& b = batches[i];
    int width = 0;
    for (int l = 0; l < h->L; ++l) width = std::max(width, h->spec.widths[l]);
    const int64_t npts = b.n_res + b.n_ic + b.n_bc;
    const int bucket = (int)std::floor(std::log2((double)std::max<int64_t>(npts, 1)));
    char key[128];
    snprintf(key, sizeof(key), "w%d_L%d_n2^%d_%s", width, h->L, bucket,
             h->spec.precision == PINN_BF16 ? "bf16" : h->spec.precision == PINN_TF32 ? "tf32" : "fp32");
    auto it = cache.find(key);
    if (it != cache.end()) {
      pinn_multi_set_config(m, i, it->second);
      continue;
    }
    // which configurations differ for this network: engines per layer under each
    int32_t eng[CFG_COUNT][PINN_MAX_HIDDEN];
    bool wide_dw = false;
    for (int c = 0; c < CFG_COUNT; ++c) {
      pinn_multi_set_config(m, i, c);
      pinn_layer_engines(h, b.n_res, b.n_ic, b.n_bc, eng[c]);
    }
    for (int l = 0; l < h->L; ++l) wide_dw = wide_dw || (eng[CFG_TC_UNFUSED][l] == 1 && h->layers[l].fout > 128);
    float best_ms[CFG_COUNT];
    for (int c = 0; c < CFG_COUNT; ++c) best_ms[c] = 1e30f;
    for (int c = 0; c < CFG_COUNT && !s; ++c) {
      bool any_tc = false, same_as_tc = true;
      for (int l = 0; l < h->L; ++l) {
        any_tc = any_tc || eng[c][l] != 0;
        same_as_tc = same_as_tc && eng[c][l] == eng[CFG_TC][l];
      }
      if (c != CFG_CUDA_CORES && !any_tc) continue;                  // tensor cores do not apply
      if (c == CFG_TC_UNFUSED && same_as_tc) continue;              // nothing fused to undo
      if (c == CFG_TC_UNFUSED_DW128 && (!wide_dw)) continue;         // every dW tile is 128 rows already
      pinn_multi_set_config(m, i, c);
      for (int rep = 0; rep < 4 && !s; ++rep) {
        cudaEventRecord(e0, st);
        s = pinn_loss_grad(h, &probs[i], &b, d_params + m->poff[i], static_cast<char*>(d_ws) + off[i], sz[i],
                           d_loss + (int64_t)i * PINN_LOSS_TERMS, d_grad + m->poff[i], st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best_ms[c] = std::min(best_ms[c], ms);
      }
    }
    int choice = 0;
    for (int c = 1; c < CFG_COUNT; ++c)
      if (best_ms[c] < best_ms[choice]) choice = c;
    if (best_ms[choice] >= 1e30f) choice = CFG_CUDA_CORES;
    pinn_multi_set_config(m, i, choice);
    cache[key] = choice;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) {
    snprintf(m->err, sizeof(m->err), "autotune: %s", pinn_status_string(s));
    return s;
  }
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "w")) {
      fputs("{\n", f);
      size_t k = 0;
      for (const auto& kv : cache)
        fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kConfigNames[kv.second],
                ++k < cache.size() ? "," : "");
      fputs("}\n", f);
      fclose(f);
    }
  }
  return PINN_OK;
}

}  // extern "C"
