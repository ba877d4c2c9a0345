// L-BFGS refinement (Sec. 2.6.5, Eqs. 22-26) over the library's loss and gradient.
//
// The history of pairs s_k = theta_{k+1} - theta_k, y_k = g_{k+1} - g_k lives on the
// device (ring buffers of FP32 vectors, FP64 scalars).  The search direction
// p = -H g comes from the two-loop recursion (Nocedal and Wright, Algorithm 7.4)
// with H_0 = gamma I, gamma = s.y / y.y of the newest pair; every dot product is an
// FP64, fixed-order reduction and every scalar stays on the device, so the recursion
// issues kernels only.  The line search (Eq. 26) is a backtracking one: the first
// lambda in 1, 1/2, 1/4, ... with L(theta + lambda p) <= L(theta) + c1 lambda g.p;
// each trial reads one loss value back to the host.  Pairs with s.y <= 0 are not
// stored, and a non-descent direction restarts from -g with an empty history.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <new>

#include "internal.h"

struct pinn_lbfgs {
  pinn_handle* h = nullptr;
  int m = 0;
  int64_t P = 0;
  float* S = nullptr;      // [m][P] ring of s pairs
  float* Y = nullptr;      // [m][P] ring of y pairs
  float* g = nullptr;      // gradient at the current parameters
  float* gnew = nullptr;   // gradient at the accepted trial point
  float* p = nullptr;      // search direction
  float* q = nullptr;      // two-loop work vector
  float* trial = nullptr;  // theta + lambda p
  double* rho = nullptr;   // [m] 1 / (y.s)
  double* alpha = nullptr; // [m]
  double* sc = nullptr;    // scalars: [0] last dot, [1] gamma, [2] coefficient, [3..10] loss terms
  double* part = nullptr;  // [64] dot partials
  int count = 0, head = 0; // pairs held, ring slot of the next pair
  bool has_g = false;
  double f = 0.0;          // loss at the current parameters
  double c1 = 1e-4;
  int max_backtracks = 30;
};

namespace {

constexpr int DOT_BLOCKS = 64;

struct Comp {   // compensated FP32 sum (TwoSum), read out in FP64
  float s = 0.f, c = 0.f;
  __device__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ double value() const { return (double)s + (double)c; }
};

__global__ void k_dot_part(const float* __restrict__ a, const float* __restrict__ b, int64_t P, double* part) {
  Comp acc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    acc.add(a[i] * b[i]);
  __shared__ double sh[8];
  double v = acc.value();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// out = sum of the partials (fixed order), then a scalar rule:
//   mode 0: sc[0] = dot
//   mode 1: alpha[i] = rho[i] dot; sc[2] = -alpha[i]           (first loop)
//   mode 2: sc[2] = alpha[i] - rho[i] dot                      (second loop)
//   mode 3: rho[i] = 1 / dot                                    (new pair)
__global__ void k_dot_final(const double* part, double* sc, double* rho, double* alpha, int i, int mode) {
  if (threadIdx.x != 0) return;
  double d = 0.0;
  for (int b = 0; b < DOT_BLOCKS; ++b) d += part[b];
  sc[0] = d;
  if (mode == 1) { alpha[i] = rho[i] * d; sc[2] = -alpha[i]; }
  if (mode == 2) sc[2] = alpha[i] - rho[i] * d;
  if (mode == 3) rho[i] = 1.0 / d;
}

// gamma = s.y / y.y from two dot results held in sc[4] (s.y) and sc[5] (y.y)
__global__ void k_gamma(double* sc) {
  if (threadIdx.x == 0) sc[2] = sc[5] > 0.0 ? sc[4] / sc[5] : 1.0;
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, int64_t P, const double* coef) {
  const float c = (float)*coef;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(c, x[i], y[i]);
}
__global__ void k_scale(float* y, const float* x, int64_t P, const double* coef, float sgn) {   // y may alias x
  const float c = sgn * (float)*coef;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = c * x[i];
}
// out = a + lam b  (host scalar)
__global__ void k_add_scaled(float* __restrict__ out, const float* __restrict__ a, const float* __restrict__ b,
                             int64_t P, float lam) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fmaf(lam, b[i], a[i]);
}
__global__ void k_sub(float* __restrict__ out, const float* __restrict__ a, const float* __restrict__ b, int64_t P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

int vec_blocks(int64_t P) { return (int)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 1024)); }

void dot(pinn_lbfgs* lb, const float* a, const float* b, int i, int mode, cudaStream_t st) {
  k_dot_part<<<DOT_BLOCKS, 256, 0, st>>>(a, b, lb->P, lb->part);
  k_dot_final<<<1, 32, 0, st>>>(lb->part, lb->sc, lb->rho, lb->alpha, i, mode);
}

int slot(const pinn_lbfgs* lb, int k) { return (lb->head - lb->count + k + lb->m) % lb->m; }   // k-th oldest pair

// p = -H g from the history (two-loop recursion).
void direction(pinn_lbfgs* lb, const float* g, float* p, cudaStream_t st) {
  const int64_t P = lb->P;
  const int nb = vec_blocks(P);
  cudaMemcpyAsync(lb->q, g, sizeof(float) * P, cudaMemcpyDeviceToDevice, st);
  for (int k = lb->count - 1; k >= 0; --k) {
    const int j = slot(lb, k);
    dot(lb, lb->S + (size_t)j * P, lb->q, j, 1, st);                  // alpha_j = rho_j s_j.q
    k_axpy<<<nb, 256, 0, st>>>(lb->q, lb->Y + (size_t)j * P, P, lb->sc + 2);   // q -= alpha_j y_j
  }
  if (lb->count > 0) {
    const int j = slot(lb, lb->count - 1);
    dot(lb, lb->S + (size_t)j * P, lb->Y + (size_t)j * P, j, 0, st);
    cudaMemcpyAsync(lb->sc + 4, lb->sc, sizeof(double), cudaMemcpyDeviceToDevice, st);
    dot(lb, lb->Y + (size_t)j * P, lb->Y + (size_t)j * P, j, 0, st);
    cudaMemcpyAsync(lb->sc + 5, lb->sc, sizeof(double), cudaMemcpyDeviceToDevice, st);
    k_gamma<<<1, 32, 0, st>>>(lb->sc);
    k_scale<<<nb, 256, 0, st>>>(p, lb->q, P, lb->sc + 2, 1.f);        // r = gamma q
  } else {
    cudaMemcpyAsync(p, lb->q, sizeof(float) * P, cudaMemcpyDeviceToDevice, st);
  }
  for (int k = 0; k < lb->count; ++k) {
    const int j = slot(lb, k);
    dot(lb, lb->Y + (size_t)j * P, p, j, 2, st);                      // coef = alpha_j - rho_j y_j.r
    k_axpy<<<nb, 256, 0, st>>>(p, lb->S + (size_t)j * P, P, lb->sc + 2);   // r += coef s_j
  }
  const double minus_one = -1.0;
  cudaMemcpyAsync(lb->sc + 2, &minus_one, sizeof(double), cudaMemcpyHostToDevice, st);
  k_scale<<<nb, 256, 0, st>>>(p, p, P, lb->sc + 2, 1.f);              // p = -r
}

pinn_status read_scalar(pinn_handle* h, const double* d, double* out, cudaStream_t st) {
  if (cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    snprintf(h->err, sizeof(h->err), "L-BFGS: %s", cudaGetErrorString(cudaGetLastError()));
    return PINN_ERR_CUDA;
  }
  return PINN_OK;
}

}  // namespace

extern "C" {

pinn_status pinn_lbfgs_create(pinn_handle* h, int history, pinn_lbfgs** out) {
  if (!h || !out || history < 1 || history > 64) return PINN_ERR_INVALID_ARG;
  *out = nullptr;
  pinn_lbfgs* lb = new (std::nothrow) pinn_lbfgs();
  if (!lb) return PINN_ERR_OOM;
  lb->h = h;
  lb->m = history;
  lb->P = h->P;
  const size_t vec = sizeof(float) * (size_t)h->P;
  bool ok = cudaMalloc(&lb->S, vec * history) == cudaSuccess && cudaMalloc(&lb->Y, vec * history) == cudaSuccess &&
            cudaMalloc(&lb->g, vec) == cudaSuccess && cudaMalloc(&lb->gnew, vec) == cudaSuccess &&
            cudaMalloc(&lb->p, vec) == cudaSuccess && cudaMalloc(&lb->q, vec) == cudaSuccess &&
            cudaMalloc(&lb->trial, vec) == cudaSuccess &&
            cudaMalloc(&lb->rho, sizeof(double) * history) == cudaSuccess &&
            cudaMalloc(&lb->alpha, sizeof(double) * history) == cudaSuccess &&
            cudaMalloc(&lb->sc, sizeof(double) * 16) == cudaSuccess &&
            cudaMalloc(&lb->part, sizeof(double) * DOT_BLOCKS) == cudaSuccess;
  if (!ok) {
    const bool oom = cudaGetLastError() == cudaErrorMemoryAllocation;
    pinn_lbfgs_destroy(lb);
    return oom ? PINN_ERR_OOM : PINN_ERR_CUDA;
  }
  *out = lb;
  return PINN_OK;
}

pinn_status pinn_lbfgs_destroy(pinn_lbfgs* lb) {
  if (!lb) return PINN_OK;
  for (void* ptr : {(void*)lb->S, (void*)lb->Y, (void*)lb->g, (void*)lb->gnew, (void*)lb->p, (void*)lb->q,
                    (void*)lb->trial, (void*)lb->rho, (void*)lb->alpha, (void*)lb->sc, (void*)lb->part})
    if (ptr) cudaFree(ptr);
  delete lb;
  return PINN_OK;
}

pinn_status pinn_lbfgs_reset(pinn_lbfgs* lb) {
  if (!lb) return PINN_ERR_INVALID_ARG;
  lb->count = lb->head = 0;
  lb->has_g = false;
  return PINN_OK;
}

pinn_status pinn_lbfgs_direction(pinn_lbfgs* lb, const float* d_g, float* d_p, void* stream) {
  if (!lb || !d_g || !d_p) return PINN_ERR_INVALID_ARG;
  direction(lb, d_g, d_p, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

pinn_status pinn_lbfgs_push_pair(pinn_lbfgs* lb, const float* d_s, const float* d_y, void* stream) {
  if (!lb || !d_s || !d_y) return PINN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vec = sizeof(float) * (size_t)lb->P;
  const int j = lb->head;
  cudaMemcpyAsync(lb->S + (size_t)j * lb->P, d_s, vec, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(lb->Y + (size_t)j * lb->P, d_y, vec, cudaMemcpyDeviceToDevice, st);
  dot(lb, lb->S + (size_t)j * lb->P, lb->Y + (size_t)j * lb->P, j, 3, st);
  lb->head = (lb->head + 1) % lb->m;
  lb->count = std::min(lb->count + 1, lb->m);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

pinn_status pinn_lbfgs_step(pinn_lbfgs* lb, const pinn_problem* prob, const pinn_batch* batch, float* d_params,
                            void* d_ws, size_t ws_bytes, double* loss_out, int* backtracks_out, void* stream) {
  if (!lb || !prob || !batch || !d_params || !d_ws) return PINN_ERR_INVALID_ARG;
  pinn_handle* h = lb->h;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t P = lb->P;
  const int nb = vec_blocks(P);
  double* dloss = lb->sc + 8;   // 8 loss terms
  pinn_status s;
  if (!lb->has_g) {
    s = pinn_loss_grad(h, prob, batch, d_params, d_ws, ws_bytes, dloss, lb->g, stream);
    if (s) return s;
    if ((s = read_scalar(h, dloss, &lb->f, st))) return s;
    lb->has_g = true;
  }
  direction(lb, lb->g, lb->p, st);
  dot(lb, lb->g, lb->p, 0, 0, st);
  double gp;
  if ((s = read_scalar(h, lb->sc, &gp, st))) return s;
  if (!(gp < 0.0)) {   // not a descent direction: restart with steepest descent
    lb->count = lb->head = 0;
    const double minus_one = -1.0;
    cudaMemcpyAsync(lb->sc + 2, &minus_one, sizeof(double), cudaMemcpyHostToDevice, st);
    k_scale<<<nb, 256, 0, st>>>(lb->p, lb->g, P, lb->sc + 2, 1.f);
    dot(lb, lb->g, lb->p, 0, 0, st);
    if ((s = read_scalar(h, lb->sc, &gp, st))) return s;
  }
  double lam = 1.0, ftrial = 0.0;
  int bt = 0;
  for (;; ++bt) {
    k_add_scaled<<<nb, 256, 0, st>>>(lb->trial, d_params, lb->p, P, (float)lam);
    s = pinn_loss(h, prob, batch, lb->trial, d_ws, ws_bytes, dloss, stream);
    if (s) return s;
    if ((s = read_scalar(h, dloss, &ftrial, st))) return s;
    if (ftrial <= lb->f + lb->c1 * lam * gp || bt + 1 >= lb->max_backtracks) break;
    lam *= 0.5;
  }
  // accept: gradient at the new point, then the new pair (s = lambda p, y = g_new - g)
  s = pinn_loss_grad(h, prob, batch, lb->trial, d_ws, ws_bytes, dloss, lb->gnew, stream);
  if (s) return s;
  if ((s = read_scalar(h, dloss, &ftrial, st))) return s;
  const double lam_d = lam;
  cudaMemcpyAsync(lb->sc + 2, &lam_d, sizeof(double), cudaMemcpyHostToDevice, st);
  k_scale<<<nb, 256, 0, st>>>(lb->q, lb->p, P, lb->sc + 2, 1.f);        // s into q
  k_sub<<<nb, 256, 0, st>>>(lb->p, lb->gnew, lb->g, P);                 // y into p
  dot(lb, lb->q, lb->p, 0, 0, st);
  double sy;
  if ((s = read_scalar(h, lb->sc, &sy, st))) return s;
  if (sy > 0.0) {
    if ((s = pinn_lbfgs_push_pair(lb, lb->q, lb->p, stream))) return s;
  }
  cudaMemcpyAsync(d_params, lb->trial, sizeof(float) * P, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(lb->g, lb->gnew, sizeof(float) * P, cudaMemcpyDeviceToDevice, st);
  lb->f = ftrial;
  if (loss_out) *loss_out = ftrial;
  if (backtracks_out) *backtracks_out = bt;
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

}  // extern "C"
