// pinn_loss_grad_static: the loss + gradient entry point for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc, or any allocator, at the
// moment they need a gradient: code running inside a host callback or a real-time
// loop where allocation may block or fail, plug-ins hosted by another runtime that
// owns the device memory pool and exposes no allocation hook to them, or
// processes whose memory budget was fixed at start-up.  They cannot provide the
// workspace that pinn_loss_grad asks for.  This entry point uses instead a
// fixed-size scratch array compiled into the library as a file-scope __device__
// variable, so it needs no allocation at call time.
//
// Costs and rules (also stated in include/pinn.h):
//   - The array is PINN_STATIC_WS_BYTES (64 MiB).  Every GPU that loads the
//     library holds it until the process exits.
//   - A batch whose workspace (pinn_workspace_bytes) exceeds it is rejected with
//     PINN_ERR_WORKSPACE before any work is queued.
//   - All calls share the one array and it keeps the previous call's contents.
//     Every value the computation reads is written earlier in the same call, so
//     nothing needs clearing between calls.  Calls whose GPU work overlaps (for
//     example on two streams) race on the array and give undefined results.
//   - The launch sequence always runs eagerly, even on a handle with
//     pinn_set_graph on: capturing and instantiating a graph would allocate.
//   - In host code g_static_ws names a host-side stand-in, not device memory, so
//     every call asks the runtime for the array's device address with the handle's
//     device current (cudaGetSymbolAddress).  The lookup allocates nothing; asking
//     on every call keeps the address right after the device's context has been
//     reset and the library's device code loaded again.  The first call on a device
//     (and the first after such a reset) makes the runtime load that code, which
//     reserves the array: make it before any stream capture.
#include <cstdio>

#include "internal.h"

namespace {

constexpr size_t kStaticWsBytes = PINN_STATIC_WS_BYTES;

__device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

}  // namespace

extern "C" pinn_status pinn_loss_grad_static(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                                             const float* d_params, double* d_loss_terms, float* d_grad,
                                             void* stream) {
  if (!h || !batch) return PINN_ERR_INVALID_ARG;
  size_t need = 0;
  pinn_status s = pinn_workspace_bytes(h, batch->n_res, batch->n_ic, batch->n_bc, &need);
  if (s) return s;
  if (need > kStaticWsBytes) {
    snprintf(h->err, sizeof(h->err),
             "batch needs %zu bytes of workspace, more than the %zu-byte static array of pinn_loss_grad_static",
             need, kStaticWsBytes);
    return PINN_ERR_WORKSPACE;
  }
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device != h->device) {
    cudaGetLastError();
    snprintf(h->err, sizeof(h->err),
             "pinn_loss_grad_static: the current device (%d) is not the device the handle was created on (%d)",
             device, h->device);
    return PINN_ERR_INVALID_ARG;
  }
  void* ws = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ws, g_static_ws);
  if (e != cudaSuccess || !ws) {
    cudaGetLastError();
    snprintf(h->err, sizeof(h->err), "pinn_loss_grad_static: cudaGetSymbolAddress of the static workspace: %s",
             cudaGetErrorString(e));
    return PINN_ERR_CUDA;
  }
  return pinn::loss_grad_eager(h, prob, batch, d_params, ws, kStaticWsBytes, d_loss_terms, d_grad, stream);
}
