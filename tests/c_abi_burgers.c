/*
 * A plain C caller of libpinn: no Python, no torch, only include/pinn.h and the CUDA
 * runtime for device memory.  It builds a 2 -> 3x32 (RWF) -> 1 Burgers network in FP32,
 * evaluates one loss + gradient on deterministic points, writes every input and the
 * result to the file named by argv[1] (the test recomputes them with the FP64 oracle),
 * then runs a few Adam steps and prints the first and last loss.
 *
 * File layout (little endian): int64 P, n_res, n_ic, n_bc; float params[P];
 * float x_res[2][n_res], x_ic[2][n_ic], g_ic[n_ic], x_bc[2][n_bc], g_bc[n_bc];
 * double loss_terms[8]; float grad[P].
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "pinn.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static double uniform01(void) {   /* 64-bit LCG (Knuth's MMIX constants), top 53 bits */
  rng_state = rng_state * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(rng_state >> 11) * (1.0 / 9007199254740992.0);
}
static double uniform(double a, double b) { return a + (b - a) * uniform01(); }

#define CHECK_PINN(call)                                                        \
  do {                                                                          \
    pinn_status s_ = (call);                                                    \
    if (s_ != PINN_OK) {                                                        \
      fprintf(stderr, "%s failed: %s\n", #call, pinn_status_string(s_));        \
      return 1;                                                                 \
    }                                                                           \
  } while (0)
#define CHECK_CUDA(call)                                                        \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));        \
      return 1;                                                                 \
    }                                                                           \
  } while (0)

static float* to_device(const float* h, size_t n) {
  float* d = NULL;
  if (cudaMalloc((void**)&d, n * sizeof(float) + 16) != cudaSuccess) return NULL;
  if (n && cudaMemcpy(d, h, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
  return d;
}

int main(int argc, char** argv) {
  if (argc < 2) {
    fprintf(stderr, "usage: %s OUTPUT_FILE\n", argv[0]);
    return 2;
  }
  pinn_spec spec = {0};
  spec.pde = PINN_BURGERS_1D;
  spec.n_hidden = 3;
  spec.widths[0] = spec.widths[1] = spec.widths[2] = 32;
  spec.ff_m = 0;
  spec.rwf = 1;
  spec.precision = PINN_FP32;
  pinn_handle* h = NULL;
  CHECK_PINN(pinn_create(&spec, &h));
  int64_t P = 0;
  CHECK_PINN(pinn_param_count(h, &P));

  const int64_t n_res = 1000, n_ic = 100, n_bc = 100;
  const double pi = 3.14159265358979323846;
  float* params = (float*)malloc((size_t)P * sizeof(float));
  for (int64_t i = 0; i < P; ++i) params[i] = (float)uniform(-0.3, 0.3);
  float* x_res = (float*)malloc(2 * n_res * sizeof(float));
  for (int64_t i = 0; i < n_res; ++i) {
    x_res[i] = (float)uniform(-1.0, 1.0);           /* x */
    x_res[n_res + i] = (float)uniform(0.0, 1.0);    /* t */
  }
  float* x_ic = (float*)malloc(2 * n_ic * sizeof(float));
  float* g_ic = (float*)malloc(n_ic * sizeof(float));
  for (int64_t i = 0; i < n_ic; ++i) {
    x_ic[i] = (float)uniform(-1.0, 1.0);
    x_ic[n_ic + i] = 0.f;
    g_ic[i] = (float)(-sin(pi * x_ic[i]));
  }
  float* x_bc = (float*)malloc(2 * n_bc * sizeof(float));
  float* g_bc = (float*)malloc(n_bc * sizeof(float));
  for (int64_t i = 0; i < n_bc; ++i) {
    x_bc[i] = (i % 2) ? 1.f : -1.f;
    x_bc[n_bc + i] = (float)uniform(0.0, 1.0);
    g_bc[i] = 0.f;
  }

  float* d_params = to_device(params, (size_t)P);
  float* d_x_res = to_device(x_res, 2 * n_res);
  float* d_x_ic = to_device(x_ic, 2 * n_ic);
  float* d_g_ic = to_device(g_ic, n_ic);
  float* d_x_bc = to_device(x_bc, 2 * n_bc);
  float* d_g_bc = to_device(g_bc, n_bc);
  if (!d_params || !d_x_res || !d_x_ic || !d_g_ic || !d_x_bc || !d_g_bc) {
    fprintf(stderr, "device allocation failed\n");
    return 1;
  }
  float *d_grad = NULL, *d_m = NULL, *d_v = NULL;
  double* d_loss = NULL;
  CHECK_CUDA(cudaMalloc((void**)&d_grad, (size_t)P * sizeof(float)));
  CHECK_CUDA(cudaMalloc((void**)&d_m, (size_t)P * sizeof(float)));
  CHECK_CUDA(cudaMalloc((void**)&d_v, (size_t)P * sizeof(float)));
  CHECK_CUDA(cudaMemset(d_m, 0, (size_t)P * sizeof(float)));
  CHECK_CUDA(cudaMemset(d_v, 0, (size_t)P * sizeof(float)));
  CHECK_CUDA(cudaMalloc((void**)&d_loss, PINN_LOSS_TERMS * sizeof(double)));

  pinn_batch batch;
  batch.x_res = d_x_res; batch.n_res = n_res;
  batch.x_ic = d_x_ic; batch.g_ic = d_g_ic; batch.n_ic = n_ic; batch.ic_mask = 1u;
  batch.x_bc = d_x_bc; batch.g_bc = d_g_bc; batch.n_bc = n_bc; batch.bc_mask = 1u;
  pinn_problem prob;
  prob.nu = 0.01 / pi;
  prob.lambda_pde = prob.lambda_ic = prob.lambda_bc = 1.0;

  size_t ws_bytes = 0;
  CHECK_PINN(pinn_workspace_bytes(h, n_res, n_ic, n_bc, &ws_bytes));
  void* d_ws = NULL;
  CHECK_CUDA(cudaMalloc(&d_ws, ws_bytes));

  CHECK_PINN(pinn_loss_grad(h, &prob, &batch, d_params, d_ws, ws_bytes, d_loss, d_grad, NULL));
  CHECK_CUDA(cudaDeviceSynchronize());
  CHECK_PINN(pinn_status_poll(h, NULL));
  double loss[PINN_LOSS_TERMS];
  float* grad = (float*)malloc((size_t)P * sizeof(float));
  CHECK_CUDA(cudaMemcpy(loss, d_loss, sizeof(loss), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(grad, d_grad, (size_t)P * sizeof(float), cudaMemcpyDeviceToHost));

  FILE* f = fopen(argv[1], "wb");
  if (!f) {
    fprintf(stderr, "cannot open %s\n", argv[1]);
    return 1;
  }
  const int64_t header[4] = {P, n_res, n_ic, n_bc};
  fwrite(header, sizeof(int64_t), 4, f);
  fwrite(params, sizeof(float), (size_t)P, f);
  fwrite(x_res, sizeof(float), 2 * n_res, f);
  fwrite(x_ic, sizeof(float), 2 * n_ic, f);
  fwrite(g_ic, sizeof(float), n_ic, f);
  fwrite(x_bc, sizeof(float), 2 * n_bc, f);
  fwrite(g_bc, sizeof(float), n_bc, f);
  fwrite(loss, sizeof(double), PINN_LOSS_TERMS, f);
  fwrite(grad, sizeof(float), (size_t)P, f);
  fclose(f);

  /* a few Adam steps through the same ABI */
  double first = loss[0], last = loss[0];
  for (int64_t step = 1; step <= 20; ++step) {
    CHECK_PINN(pinn_adam_step(d_params, d_grad, d_m, d_v, P, step, 1e-3f, 0.9f, 0.999f, 1e-8f, NULL));
    CHECK_PINN(pinn_loss_grad(h, &prob, &batch, d_params, d_ws, ws_bytes, d_loss, d_grad, NULL));
  }
  CHECK_CUDA(cudaMemcpy(loss, d_loss, sizeof(loss), cudaMemcpyDeviceToHost));
  CHECK_PINN(pinn_status_poll(h, NULL));
  last = loss[0];
  printf("{\"loss_first\": %.17g, \"loss_last\": %.17g, \"P\": %lld}\n", first, last, (long long)P);

  cudaFree(d_ws); cudaFree(d_loss); cudaFree(d_v); cudaFree(d_m); cudaFree(d_grad);
  cudaFree(d_g_bc); cudaFree(d_x_bc); cudaFree(d_g_ic); cudaFree(d_x_ic); cudaFree(d_x_res); cudaFree(d_params);
  free(grad); free(g_bc); free(x_bc); free(g_ic); free(x_ic); free(x_res); free(params);
  CHECK_PINN(pinn_destroy(h));
  return 0;
}
