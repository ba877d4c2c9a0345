// C ABI entry points of libpinn: validation, workspace planning and the launch
// sequence of one loss / loss+gradient evaluation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"
#include "tc.h"

using namespace pinn;

namespace {

void set_err(pinn_handle* h, const char* fmt, ...) {
  if (!h) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(h->err, sizeof(h->err), fmt, ap);
  va_end(ap);
}

pinn_status cuda_check(pinn_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PINN_OK;
  set_err(h, "%s: %s", what, cudaGetErrorString(e));
  return PINN_ERR_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int PROF_MAX = 16384;
enum Phase { PH_RWF = 0, PH_EMBED = 1, PH_FWD = 2, PH_OUT = 3, PH_DW = 4, PH_ADJ = 5, PH_RED = 6, PH_OTHER = 7,
             PH_ADJDW = 8 };

// Brackets one launch group with a pair of CUDA events when profiling is on.
struct PhaseScope {
  pinn_handle* h;
  cudaStream_t st;
  int idx = -1;
  PhaseScope(pinn_handle* hh, cudaStream_t s, int phase, int launches) : h(hh), st(s) {
    if (!h->prof) return;
    if (h->prof_n >= PROF_MAX) { ++h->prof_dropped; return; }
    idx = h->prof_n++;
    h->prof_phase[idx] = phase;
    h->prof_launches[idx] = launches;
    cudaEventRecord(h->prof_ev[2 * idx], st);
  }
  ~PhaseScope() {
    if (idx >= 0) cudaEventRecord(h->prof_ev[2 * idx + 1], st);
  }
};

int pde_din(int pde) { return pde == PINN_MAXWELL_TE_2D ? 3 : 2; }
int pde_dout(int pde) { return (pde == PINN_NS_STEADY_2D || pde == PINN_MAXWELL_TE_2D) ? 3 : 1; }

}  // namespace

namespace pinn {

pinn_status make_plan(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, Plan* p) {
  Plan q;
  q.n_res = n_res; q.n_ic = n_ic; q.n_bc = n_bc;
  q.ncols = 4 * (n_res + n_ic + n_bc);
  q.NP = (int64_t)align_up((size_t)std::max<int64_t>(n_res + n_ic + n_bc, 1), PT_ALIGN);
  q.NC = 4 * q.NP;
  q.es = (h->spec.precision == PINN_BF16) ? 2 : 4;
  q.lo = (h->spec.precision == PINN_BF16);
  q.lo_es = 2;
  const int L = h->L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  q.nbpart = (int)std::min<int64_t>(256, std::max<int64_t>(1, q.NC / 1024));   // row-reduction chunks of >= 256 points
  if (h->spec.ff_m) {
    q.A[0] = take((size_t)2 * h->spec.ff_m * q.NC * q.es);
    if (q.lo) q.Alo[0] = take((size_t)2 * h->spec.ff_m * q.NP * q.lo_es);
  }
  // One jet array per layer: the activations A_l.  The pre-activations Z_l are not
  // kept: the adjoint epilogues recompute t', t'', t''' from A_l.
  for (int l = 1; l <= L; ++l) {
    q.A[l] = take((size_t)h->spec.widths[l - 1] * q.NC * q.es);
    if (q.lo) q.Alo[l] = take((size_t)h->spec.widths[l - 1] * q.NP * q.lo_es);
    // the sine activation's adjoint needs z itself (cos(w z) is not a function of sin(w z))
    if (h->act == PINN_ACT_SINE) q.Z[l] = take((size_t)h->spec.widths[l - 1] * q.NC * 4);
  }
  // the ping-pong adjoints also hold the input-jet adjoint (2m rows) of pinn_loss_grad_ff
  const size_t zrows = (size_t)std::max(h->w_max, 2 * h->spec.ff_m);
  q.Zbar[0] = take(zrows * q.NC * q.es);
  q.Zbar[1] = take(zrows * q.NC * q.es);
  q.nloss_blocks = out_loss_tma_ok(h->spec.precision, h->act, h->spec.widths[L - 1])
                      ? out_loss_tma_blocks(q.NP, h->sm_count)
                      : out_loss_blocks(q.NP);
  q.losspart = take((size_t)q.nloss_blocks * 8 * sizeof(double));
  if (h->causal_M > 0) q.segpart = take((size_t)q.nloss_blocks * CAUSAL_MAX * 4 * sizeof(double));
  if (h->spec.ff_m) q.ffpart = take((size_t)h->spec.ff_m * FFG_BLOCKS * h->d_in * sizeof(double));
  *p = q;
  p->total = off;
  return PINN_OK;
}

}  // namespace pinn

// Per-call layer plan (weights and split partials live in the workspace too).
namespace {

struct CallPlan {
  Plan p;
  LayerPlan lay[PINN_MAX_HIDDEN + 1];
  bool tc[PINN_MAX_HIDDEN + 1];      // layer li runs its jet GEMMs on tensor cores
  bool fused[PINN_MAX_HIDDEN + 1];   // layer li's adjoint and weight gradient run as one fused kernel
  bool fused_db[PINN_MAX_HIDDEN + 1];  // layer li's bias partials come from a fused adjoint epilogue
  bool out_db = false;                 // the last hidden layer's bias partials come from the output/loss kernel
  int nbpart[PINN_MAX_HIDDEN + 1];     // bias partial count of layer li
  bool pm = false;                     // TF32 on tensor cores: point-major operand copies
  size_t apm[2] = {0, 0};              // point-major A_l, buffer l % 2 ([NC][fin] FP32)
  size_t zbpm[2] = {0, 0};             // point-major adjoints, ping-pong like Zbar
};

pinn_status plan_call(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, CallPlan* c) {
  make_plan(h, n_res, n_ic, n_bc, &c->p);
  size_t off = c->p.total;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const int L1 = h->L + 1;
  for (int li = 0; li < L1; ++li) {
    const bool raw = (li == 0 && !h->spec.ff_m);
    c->tc[li] = li < h->L && !raw && tc_layer_supported(h, li, c->p.NC);
  }
  if (h->spec.precision == PINN_TF32) {
    // TF32 tensor-core layers hand point-major operands to each other: all or none
    bool all = true;
    for (int li = h->first_gemm; li < h->L; ++li) all = all && c->tc[li];
    for (int li = 0; li < L1; ++li) c->tc[li] = c->tc[li] && all;
    c->pm = all && h->first_gemm < h->L;
  }
  for (int li = 0; li < L1; ++li) c->fused[li] = c->tc[li] && tc_adjdw_supported(h, li, c->p.NC);
  for (int li = 0; li < L1; ++li) {
    LayerPlan lp = h->layers[li];
    const bool raw = (li == 0 && !h->spec.ff_m);
    lp.w32 = take((size_t)lp.fin * lp.fout * 4);
    lp.wc = take((size_t)lp.fin * lp.fout * c->p.es);
    lp.wtc = take((size_t)lp.fin * lp.fout * c->p.es);
    lp.wt32 = take((size_t)lp.fin * lp.fout * 4);
    lp.wlo = take((size_t)lp.fin * lp.fout * c->p.es);
    if (raw) {
      lp.nsplit = 0;
    } else if (li == h->L) {
      lp.nsplit = c->p.nloss_blocks;   // output layer: one dW partial per output/loss block
    } else if (c->fused[li]) {
      lp.nsplit = tc_adjdw_splits(h, lp.fin, c->p.NC);   // one partial per fused-kernel CTA and m-tile
    } else if (c->tc[li]) {
      lp.nsplit = tc_dw_splits(h, lp.fout, lp.fin, c->p.NC);
    } else {
      const int tiles = ((lp.fout + 63) / 64) * ((lp.fin + 63) / 64);
      int ns = (4 * std::max(h->sm_count, 1) + tiles - 1) / tiles;
      ns = (int)std::max<int64_t>(1, std::min<int64_t>(ns, c->p.NC / 128));   // >= 128 jet columns per split
      lp.nsplit = ns;
    }
    // the output layer keeps room for its compacted partials after the per-block ones
    const int slots = std::max(lp.nsplit, 0) + (li == h->L ? OUT_SUM_SLOTS : 0);
    lp.dwpart = take((size_t)slots * lp.fout * lp.fin * 4);
    // Bias partials of hidden layer li come from the tensor-core adjoint epilogue of
    // layer li+1 when that one runs on tensor cores, else from a row reduction.
    c->fused_db[li] = (li + 1 < h->L) && c->tc[li + 1];
    // the last hidden layer's bias partials come from the output/loss kernel (it
    // writes that layer's adjoint), unless it is a first layer on raw coordinates
    const bool out_db = (li == h->L - 1) && !raw;
    if (li == h->L - 1) c->out_db = out_db;
    c->nbpart[li] = (li == h->L || out_db) ? c->p.nloss_blocks
                    : c->fused_db[li] ? (int)(c->p.NC / TC_BN) * TC_DB_PARTS : c->p.nbpart;
    const int dbs = raw ? 1 + h->d_in : 1;
    lp.dbpart = take((size_t)c->nbpart[li] * lp.fout * dbs * 4);
    lp.wtlo = take((size_t)lp.fin * lp.fout * c->p.es);
    c->lay[li] = lp;
  }
  if (c->pm) {
    int fin_max = 0;
    for (int li = h->first_gemm; li < h->L; ++li) fin_max = std::max(fin_max, h->layers[li].fin);
    for (int k = 0; k < 2; ++k) c->apm[k] = take((size_t)fin_max * c->p.NC * 4);
    for (int k = 0; k < 2; ++k) c->zbpm[k] = take((size_t)h->w_max * c->p.NC * 4);
  }
  c->p.total = off;
  return PINN_OK;
}

pinn_status validate_batch(pinn_handle* h, const pinn_batch* b) {
  if (!b) { set_err(h, "batch is NULL"); return PINN_ERR_INVALID_ARG; }
  if (b->n_res < 0 || b->n_ic < 0 || b->n_bc < 0) { set_err(h, "negative point count"); return PINN_ERR_INVALID_ARG; }
  if (b->n_res + b->n_ic + b->n_bc == 0) { set_err(h, "empty batch"); return PINN_ERR_INVALID_ARG; }
  if (b->n_res > ((int64_t)1 << 34) || b->n_ic > ((int64_t)1 << 34) || b->n_bc > ((int64_t)1 << 34)) {
    set_err(h, "point count too large"); return PINN_ERR_INVALID_ARG;
  }
  if (b->n_res && !b->x_res) { set_err(h, "x_res is NULL"); return PINN_ERR_INVALID_ARG; }
  if (b->n_ic && (!b->x_ic || (b->ic_mask && !b->g_ic))) { set_err(h, "initial-set pointer is NULL"); return PINN_ERR_INVALID_ARG; }
  if (b->n_bc && (!b->x_bc || (b->bc_mask && !b->g_bc))) { set_err(h, "boundary-set pointer is NULL"); return PINN_ERR_INVALID_ARG; }
  if ((b->ic_mask | b->bc_mask) >> h->d_out) { set_err(h, "mask names an output the network does not have"); return PINN_ERR_INVALID_ARG; }
  return PINN_OK;
}

// How one call is split into passes over point chunks, and what each pass adds to.
struct PassCtx {
  int64_t N_res, N_ic, N_bc;   // the batch's full counts: every mean is normalised by these
  bool first, last;            // first pass starts the loss/gradient sums; last one writes the loss
  double* loss_acc;            // 5 FP64 running loss sums (chunked calls only)
};

// One forward + reverse sweep over the points of `b` (the whole batch, or one chunk),
// in stages: the prologue (RWF weights, input jets), one forward stage per GEMM layer,
// then per loss term the output stage, one backward stage per hidden layer (top down)
// and the gradient finalisation.  run_pass runs the stages in this order; the
// many-network step runs the stages of all its networks level by level, so that their
// tensor-core GEMMs of one level share grouped launches.
struct Pass {
  pinn_handle* h = nullptr;
  const pinn_problem* prob = nullptr;
  const pinn_batch* b = nullptr;
  const float* d_params = nullptr;
  char* ws = nullptr;
  double* d_loss = nullptr;
  float* d_grad = nullptr;
  bool want_grad = false;
  PassCtx pc{};
  float* d_grad_terms = nullptr;   // per-term gradients [3][P] (Sec. 2.6.4), or null
  float* d_grad_ff = nullptr;      // input-map gradient, or null
  CallPlan cp;
  // the loss term of the output, backward and finalisation stages
  int term = 0;
  double lam_pde = 0, lam_ic = 0, lam_bc = 0;
  float* grad_out = nullptr;
  OutArgs oa{};

  int nterms() const { return d_grad_terms ? 3 : 1; }
  const float* W32(int li) const { return reinterpret_cast<const float*>(ws + cp.lay[li].w32); }
  const float* bias(int li) const { return d_params + cp.lay[li].off_b; }

  pinn_status init(size_t ws_bytes) {
    plan_call(h, b->n_res, b->n_ic, b->n_bc, &cp);
    if (ws_bytes < cp.p.total) {
      set_err(h, "workspace too small: %zu < %zu bytes", ws_bytes, cp.p.total); return PINN_ERR_WORKSPACE;
    }
    return PINN_OK;
  }

  // 1-2: RWF weights and the input jets.
  pinn_status prologue(cudaStream_t st) {
    const Plan& p = cp.p;
    const int L1 = h->L + 1, prec = h->spec.precision, mode = h->jet_mode;
    const bool sine = h->act == PINN_ACT_SINE;
    // 1. RWF weights (Eq. 15) for every layer.
    RwfArgs ra{};
    ra.params = d_params; ra.ws = ws; ra.L1 = L1; ra.rwf = h->spec.rwf; ra.prec = prec;
    for (int li = 0; li < L1; ++li) {
      ra.fin[li] = cp.lay[li].fin; ra.fout[li] = cp.lay[li].fout;
      ra.offV[li] = cp.lay[li].off_V; ra.offs[li] = cp.lay[li].off_s;
      ra.w32[li] = cp.lay[li].w32; ra.wc[li] = cp.lay[li].wc; ra.wtc[li] = cp.lay[li].wtc;
      ra.wt32[li] = cp.lay[li].wt32; ra.wlo[li] = cp.lay[li].wlo; ra.wtlo[li] = cp.lay[li].wtlo;
    }
    { PhaseScope ps(h, st, PH_RWF, 1); launch_rwf_prep(ra, st); }

    // 2. Input embedding jets (Eq. 14) or the first layer on raw coordinates.
    PhaseScope ps(h, st, PH_EMBED, 1);
    if (h->spec.ff_m) {
      launch_embed_ff(b->x_res, b->x_ic, b->x_bc, b->n_res, b->n_ic, b->n_bc, h->d_in, h->ff_B, h->spec.ff_m, mode,
                      ws + p.A[0], p.lo ? ws + p.Alo[0] : nullptr, p.NP, prec, st);
    } else {
      launch_first_layer(b->x_res, b->x_ic, b->x_bc, b->n_res, b->n_ic, b->n_bc, h->d_in, W32(0), bias(0),
                         cp.lay[0].fout, mode, ws + p.A[1], p.lo ? ws + p.Alo[1] : nullptr, p.NP, prec, h->omega0,
                         sine ? reinterpret_cast<float*>(ws + p.Z[1]) : nullptr, st);
    }
    if (cp.pm) {
      const int f0 = h->first_gemm;
      launch_to_point_major(ws + p.A[f0], ws + cp.apm[f0 % 2], cp.lay[f0].fin, p.NC, st);
    }
    return PINN_OK;
  }

  // 3. Hidden jet GEMM li (first_gemm <= li < L) with the tanh-jet epilogue.
  pinn_status forward(int li, cudaStream_t st) {
    const Plan& p = cp.p;
    const int L = h->L, prec = h->spec.precision;
    const bool sine = h->act == PINN_ACT_SINE;
    EpiArgs e{};
    e.bias = bias(li); e.out = ws + p.A[li + 1];
    e.alo_out = p.lo ? ws + p.Alo[li + 1] : nullptr;
    // BF16 storage is rounded, so consumers add the low half back; TF32 storage is
    // exact FP32 and only the tensor-core forward (which truncates) uses the low half.
    e.alo_in = (p.lo && prec == PINN_BF16) ? ws + p.Alo[li] : nullptr;
    e.jet_mode = h->jet_mode;
    e.act = h->act; e.omega0 = h->omega0;
    e.zout = sine ? reinterpret_cast<float*>(ws + p.Z[li + 1]) : nullptr;
    // alternate the tile order from layer to layer: each forward starts on the tiles
    // the previous kernel wrote last (the embedding goes first to last)
    e.reverse = ((li - h->first_gemm) % 2 == 0) ? 1 : 0;
    PhaseScope ps(h, st, PH_FWD, 1);
    if (cp.tc[li] && cp.pm) {
      // TF32: point-major input; the epilogue also writes the next layer's point-major input
      e.out_pm = (li + 1 < L) ? ws + cp.apm[(li + 1) % 2] : nullptr;
      return tc_gemm_fwd(h, ws + cp.lay[li].wc, ws + cp.lay[li].wlo, ws + cp.apm[li % 2], nullptr, cp.lay[li].fout,
                         cp.lay[li].fin, p.NC, e, st);
    }
    if (cp.tc[li])
      return tc_gemm_fwd(h, ws + cp.lay[li].wc, ws + cp.lay[li].wlo, ws + p.A[li], ws + p.Alo[li], cp.lay[li].fout,
                         cp.lay[li].fin, p.NC, e, st);
    launch_simt_gemm_fwd(W32(li), ws + p.A[li], cp.lay[li].fout, cp.lay[li].fin, p.NP, e, prec, st);
    return PINN_OK;
  }

  // 4-5 for loss term t (one weighted term, or term t of the per-term gradients):
  // output layer, residual, loss partials, adjoint seed and Zbar_L; then the output
  // layer's dW partials compacted.  Without a gradient the pass ends here.
  pinn_status output(int t, cudaStream_t st) {
    const Plan& p = cp.p;
    const int L = h->L, prec = h->spec.precision, mode = h->jet_mode;
    const bool sine = h->act == PINN_ACT_SINE;
    term = t;
    lam_pde = d_grad_terms ? (term == 0 ? 1.0 : 0.0) : prob->lambda_pde;
    lam_ic = d_grad_terms ? (term == 1 ? 1.0 : 0.0) : prob->lambda_ic;
    lam_bc = d_grad_terms ? (term == 2 ? 1.0 : 0.0) : prob->lambda_bc;
    grad_out = d_grad_terms ? d_grad_terms + (size_t)term * h->P : d_grad;

    // 4. Output layer, residual, loss partials, adjoint seed and Zbar_L.
    oa = OutArgs{};
    oa.AL = ws + p.A[L]; oa.ALlo = (p.lo && prec == PINN_BF16) ? ws + p.Alo[L] : nullptr;
    oa.W = W32(L); oa.b = bias(L);
    oa.g_ic = b->g_ic; oa.g_bc = b->g_bc; oa.ic_mask = b->ic_mask; oa.bc_mask = b->bc_mask;
    oa.n_res = p.n_res; oa.n_ic = p.n_ic; oa.n_bc = p.n_bc; oa.NP = p.NP; oa.NC = p.NC;
    oa.w = cp.lay[L].fin; oa.d_out = h->d_out; oa.pde = h->spec.pde; oa.jet_mode = mode;
    oa.nu = (float)prob->nu;
    oa.k_pde = pc.N_res ? (float)(lam_pde / (double)pc.N_res) : 0.f;
    oa.k_ic = pc.N_ic ? (float)(lam_ic / (double)pc.N_ic) : 0.f;
    oa.k_bc = pc.N_bc ? (float)(lam_bc / (double)pc.N_bc) : 0.f;
    oa.want_grad = want_grad;
    oa.x_res = b->x_res;
    oa.dwpart = reinterpret_cast<float*>(ws + cp.lay[L].dwpart);
    oa.dbpart = reinterpret_cast<float*>(ws + cp.lay[L].dbpart);
    oa.dbhid = cp.out_db ? reinterpret_cast<float*>(ws + cp.lay[L - 1].dbpart) : nullptr;
    oa.Zbar = ws + p.Zbar[L % 2];
    oa.ZL = sine ? reinterpret_cast<const float*>(ws + p.Z[L]) : nullptr;
    oa.reverse = ((L - 1 - h->first_gemm) % 2 == 0) ? 0 : 1;   // against the last forward's order
    oa.omega0 = h->omega0;
    oa.losspart = reinterpret_cast<double*>(ws + p.losspart);
    oa.status = h->d_status;
    const bool causal = h->causal_M > 0;
    double* causal_omega = h->d_scratch + 256;                           // [CAUSAL_MAX] doubles
    float* causal_scale = reinterpret_cast<float*>(h->d_scratch + 288);   // [CAUSAL_MAX] floats
    if (causal) {
      // Temporal causality (Sec. 2.6.8): a first pass gathers the segment losses, the
      // weights follow, and the seeds of the second pass are scaled per segment.
      oa.segments = h->causal_M;
      oa.t_index = h->spec.pde == PINN_MAXWELL_TE_2D ? 2 : 1;
      oa.t0 = (float)h->causal_t0;
      oa.tinv = (float)(h->causal_M / (h->causal_t1 - h->causal_t0));
      if (term == 0) {
        OutArgs o1 = oa;
        o1.want_grad = 0;
        o1.segpart = reinterpret_cast<double*>(ws + p.segpart);
        PhaseScope ps(h, st, PH_OUT, 1);
        const cudaError_t e = launch_out_loss(o1, prec, p.nloss_blocks, st);
        if (e != cudaSuccess) return cuda_check(h, e, "output/loss launch");
        launch_finalize_causal(o1.segpart, o1.losspart, p.nloss_blocks, h->causal_M, h->causal_eps,
                               b->ic_mask ? pc.N_ic : 0, b->bc_mask ? pc.N_bc : 0, prob->lambda_pde,
                               prob->lambda_ic, prob->lambda_bc, lam_pde, d_loss, causal_omega, causal_scale,
                               h->d_status, st);
      }
      oa.seg_scale = lam_pde != 0.0 ? causal_scale : nullptr;
    }
    if (!causal || want_grad) {
      PhaseScope ps(h, st, PH_OUT, 1);
      const cudaError_t e = launch_out_loss(oa, prec, p.nloss_blocks, st);
      if (e != cudaSuccess) return cuda_check(h, e, "output/loss launch");
    }
    if (term == 0 && !causal) {   // the loss terms are unweighted sums; the total uses the problem's weights
      PhaseScope ps_fl(h, st, PH_RED, 1);
      launch_finalize_loss(oa.losspart, p.nloss_blocks, pc.N_res, (b->ic_mask ? pc.N_ic : 0),
                           (b->bc_mask ? pc.N_bc : 0), prob->lambda_pde, prob->lambda_ic, prob->lambda_bc, d_loss,
                           pc.loss_acc, pc.first, pc.last, h->d_status, st);
    }
    if (!want_grad) return PINN_OK;
    if (cp.pm) {
      PhaseScope ps(h, st, PH_OTHER, 1);
      launch_to_point_major(ws + p.Zbar[L % 2], ws + cp.zbpm[L % 2], cp.lay[L].fin, p.NC, st);
    }

    // 5. The output layer's dW and bias partials came from the output/loss kernel; its
    //    per-block dW partials are compacted (in order) so the finalisation reads a few.
    PhaseScope ps(h, st, PH_RED, 1);
    const LayerPlan& lo = cp.lay[L];
    float* part = reinterpret_cast<float*>(ws + lo.dwpart);
    launch_sum_splits(part, part + (size_t)lo.nsplit * lo.fout * lo.fin, lo.nsplit, OUT_SUM_SLOTS,
                      (int64_t)lo.fout * lo.fin, st);
    return PINN_OK;
  }

  // 6. Hidden layer li (L-1 down to 0): dW, db, then the adjoint GEMM into the layer below.
  pinn_status backward(int li, cudaStream_t st) {
    const Plan& p = cp.p;
    const int L = h->L, prec = h->spec.precision, mode = h->jet_mode;
    const bool sine = h->act == PINN_ACT_SINE;
    pinn_status s = PINN_OK;
    const LayerPlan& lp = cp.lay[li];
    void* zb = ws + p.Zbar[(li + 1) % 2];
    const bool raw = (li == 0 && !h->spec.ff_m);
    if (!raw && !cp.fused[li]) {   // (a fused layer's weight gradient comes with its adjoint below)
      PhaseScope ps(h, st, PH_DW, 1);
      if (cp.tc[li]) {
        s = tc_gemm_dw(h, zb, ws + p.A[li], lp.fout, lp.fin, p.NC, lp.nsplit, reinterpret_cast<float*>(ws + lp.dwpart),
                       st);
        if (s) return s;
      } else {
        launch_simt_gemm_dw(zb, false, ws + p.A[li], false, lp.fout, lp.fin, p.NC, lp.nsplit,
                            reinterpret_cast<float*>(ws + lp.dwpart), prec, st);
      }
    }
    if (!cp.fused_db[li] && !(li == L - 1 && cp.out_db)) {
      PhaseScope ps(h, st, PH_RED, 1);
      launch_row_reduce(zb, false, lp.fout, p.NP, p.n_res, p.n_ic, p.n_bc, p.nbpart, b->x_res, b->x_ic, b->x_bc,
                        raw ? h->d_in : 0, mode, reinterpret_cast<float*>(ws + lp.dbpart), prec, st);
    }
    if (li == 0 && d_grad_ff) {
      // Input-map gradient: Abar_0 = W_1^T Zbar_1 (into the free adjoint buffer), then
      // its contraction with the embedding's derivatives by B (or the periods).
      PhaseScope ps(h, st, PH_OTHER, 3);
      double* ffpart = reinterpret_cast<double*>(ws + p.ffpart);
      launch_simt_gemm_lin(reinterpret_cast<const float*>(ws + lp.wt32), zb, lp.fin, lp.fout, p.NP, ws + p.Zbar[0],
                           prec, st);
      launch_ff_grad(ws + p.Zbar[0], b->x_res, b->x_ic, b->x_bc, p.n_res, p.n_ic, p.n_bc, h->d_in, h->ff_B,
                     h->spec.ff_m, mode, p.NP, ffpart, prec, st);
      launch_ff_grad_final(ffpart, h->d_in, h->spec.ff_m, h->periodic, h->periods, pc.first ? 0 : 1, d_grad_ff, st);
    }
    if (li < 1) return PINN_OK;
    EpiArgs e{};
    e.out = ws + p.Zbar[li % 2]; e.ain = ws + p.A[li];
    e.ain_lo = p.lo ? ws + p.Alo[li] : nullptr;
    e.jet_mode = mode;
    e.act = h->act; e.omega0 = h->omega0;
    e.zin = sine ? reinterpret_cast<const float*>(ws + p.Z[li]) : nullptr;
    // against the order in which the adjoint it reads was written
    e.reverse = (((L - 1 - li) % 2 == 0) == (oa.reverse != 0)) ? 0 : 1;
    if (cp.fused_db[li - 1]) {
      e.dbpart = reinterpret_cast<float*>(ws + cp.lay[li - 1].dbpart);
      e.dterms = (li - 1 == 0 && !h->spec.ff_m) ? h->d_in : 0;
      e.x_res = b->x_res; e.x_ic = b->x_ic; e.x_bc = b->x_bc;
      e.n_res = p.n_res; e.n_ic = p.n_ic; e.n_bc = p.n_bc;
    }
    PhaseScope ps(h, st, cp.fused[li] ? PH_ADJDW : PH_ADJ, 1);
    if (cp.fused[li])
      return tc_gemm_adjdw(h, ws + lp.wtc, zb, ws + p.A[li], lp.fin, lp.fout, p.NC, e,
                           reinterpret_cast<float*>(ws + lp.dwpart), lp.nsplit, st);
    if (cp.tc[li] && cp.pm) {
      e.out_pm = (li - 1 >= 1) ? ws + cp.zbpm[li % 2] : nullptr;
      return tc_gemm_adj(h, ws + lp.wtc, ws + lp.wtlo, ws + cp.zbpm[(li + 1) % 2], lp.fin, lp.fout, p.NC, e, st);
    }
    if (cp.tc[li]) return tc_gemm_adj(h, ws + lp.wtc, nullptr, zb, lp.fin, lp.fout, p.NC, e, st);
    launch_simt_gemm_adj(reinterpret_cast<const float*>(ws + lp.wt32), zb, lp.fin, lp.fout, p.NP, e, prec, st);
    return PINN_OK;
  }

  // 7. Ordered FP64 reduction + RWF chain rule into the packed gradient.
  pinn_status finalize(cudaStream_t st) {
    const Plan& p = cp.p;
    const int L = h->L, L1 = L + 1;
    FinalizeArgs fa{};
    fa.params = d_params; fa.grad = grad_out; fa.ws = ws; fa.L1 = L1; fa.rwf = h->spec.rwf;
    fa.first_raw = !h->spec.ff_m; fa.nbpart = p.nbpart; fa.accumulate = pc.first ? 0 : 1;
    for (int li = 0; li < L1; ++li) {
      fa.fin[li] = cp.lay[li].fin; fa.fout[li] = cp.lay[li].fout;
      fa.offV[li] = cp.lay[li].off_V; fa.offs[li] = cp.lay[li].off_s; fa.offb[li] = cp.lay[li].off_b;
      fa.w32[li] = cp.lay[li].w32; fa.dwpart[li] = cp.lay[li].dwpart; fa.dbpart[li] = cp.lay[li].dbpart;
      fa.nsplit[li] = cp.lay[li].nsplit;
      if (li == L) {   // the compacted output-layer partials
        fa.dwpart[li] += (size_t)cp.lay[li].nsplit * cp.lay[li].fout * cp.lay[li].fin * 4;
        fa.nsplit[li] = OUT_SUM_SLOTS;
      }
      fa.nbpart_l[li] = cp.nbpart[li];
      fa.dbstride[li] = (li == 0 && fa.first_raw) ? 1 + h->d_in : 1;
    }
    PhaseScope ps(h, st, PH_RED, 1);
    launch_finalize_grad(fa, st);
    return PINN_OK;
  }
};

pinn_status run_pass(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                     char* ws, size_t ws_bytes, double* d_loss, float* d_grad, cudaStream_t st, bool want_grad,
                     const PassCtx& pc, float* d_grad_terms = nullptr, float* d_grad_ff = nullptr) {
  Pass ps;
  ps.h = h; ps.prob = prob; ps.b = b; ps.d_params = d_params; ps.ws = ws; ps.d_loss = d_loss; ps.d_grad = d_grad;
  ps.want_grad = want_grad; ps.pc = pc; ps.d_grad_terms = d_grad_terms; ps.d_grad_ff = d_grad_ff;
  pinn_status s = ps.init(ws_bytes);
  if (s) return s;
  s = ps.prologue(st);
  for (int li = h->first_gemm; li < h->L && !s; ++li) s = ps.forward(li, st);
  if (s) return s;
  // 4-7 run once for the weighted loss, or once per loss term (weight 1 for that term,
  // 0 for the others) when the per-term gradients are asked for (Sec. 2.6.4); the
  // forward jets above are shared.
  for (int term = 0; term < ps.nterms(); ++term) {
    s = ps.output(term, st);
    if (s) return s;
    if (!want_grad) return cuda_check(h, cudaGetLastError(), "loss launch");
    for (int li = h->L - 1; li >= 0 && !s; --li) s = ps.backward(li, st);
    if (!s) s = ps.finalize(st);
    if (s) return s;
  }
  return cuda_check(h, cudaGetLastError(), "loss_grad launch");
}

// Staging area of a chunked call: the loss accumulator, then compact copies of one
// chunk's coordinates and targets, then the chunk's own pass workspace.
struct ChunkLayout {
  int64_t C = 0;                       // points per chunk
  size_t acc = 0, x_res = 0, x_ic = 0, g_ic = 0, x_bc = 0, g_bc = 0;
  size_t pass = 0;                     // offset of the pass workspace
};

ChunkLayout chunk_layout(const pinn_handle* h, int64_t C) {
  ChunkLayout c;
  c.C = C;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  c.acc = take(8 * sizeof(double));
  c.x_res = take((size_t)h->d_in * C * 4);
  c.x_ic = take((size_t)h->d_in * C * 4);
  c.g_ic = take((size_t)h->d_out * C * 4);
  c.x_bc = take((size_t)h->d_in * C * 4);
  c.g_bc = take((size_t)h->d_out * C * 4);
  c.pass = off;
  return c;
}

// Point range [s, e) of the concatenated order (interior, initial, boundary) split per set.
struct ChunkRange { int64_t r0, nr, i0, ni, b0, nb; };
ChunkRange chunk_range(int64_t s, int64_t e, int64_t n_res, int64_t n_ic, int64_t n_bc) {
  auto clip = [](int64_t s, int64_t e, int64_t lo, int64_t n, int64_t& start, int64_t& cnt) {
    const int64_t a = std::max(s, lo), b = std::min(e, lo + n);
    start = a - lo;
    cnt = std::max<int64_t>(0, b - a);
  };
  ChunkRange r;
  clip(s, e, 0, n_res, r.r0, r.nr);
  clip(s, e, n_res, n_ic, r.i0, r.ni);
  clip(s, e, n_res + n_ic, n_bc, r.b0, r.nb);
  return r;
}

size_t chunked_bytes(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc) {
  const int64_t C = h->chunk_points, N = n_res + n_ic + n_bc;
  const ChunkLayout cl = chunk_layout(h, C);
  size_t need = 0;
  for (int64_t s = 0; s < N; s += C) {
    const ChunkRange r = chunk_range(s, std::min(N, s + C), n_res, n_ic, n_bc);
    CallPlan cp;
    plan_call(h, r.nr, r.ni, r.nb, &cp);
    need = std::max(need, cp.p.total);
  }
  return cl.pass + need;
}

// Copy rows [start, start + cnt) of a [rows][ld] FP32 array into a compact [rows][cnt] one.
cudaError_t copy_rows(float* dst, const float* src, int rows, int64_t ld, int64_t start, int64_t cnt, cudaStream_t st) {
  if (cnt == 0 || rows == 0 || !src) return cudaSuccess;
  return cudaMemcpy2DAsync(dst, (size_t)cnt * 4, src + start, (size_t)ld * 4, (size_t)cnt * 4, (size_t)rows,
                           cudaMemcpyDeviceToDevice, st);
}

// Argument and state checks of one call; the mean normalisation of its pass(es).
pinn_status check_call(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                       void* d_ws, double* d_loss, float* d_grad, bool want_grad, float* d_grad_terms, PassCtx* pc) {
  if (!h) return PINN_ERR_INVALID_ARG;
  if (!prob || !d_params || !d_ws || !d_loss || (want_grad && !d_grad && !d_grad_terms)) {
    set_err(h, "NULL argument"); return PINN_ERR_INVALID_ARG;
  }
  if (reinterpret_cast<uintptr_t>(d_ws) % 256) { set_err(h, "workspace must be 256-byte aligned"); return PINN_ERR_INVALID_ARG; }
  {
    // every buffer the handle owns (status word, scratch) lives on the device it was
    // created on; kernels launched with another device current could not reach them
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
      cudaGetLastError();
      set_err(h, "the current device (%d) is not the device the handle was created on (%d)", dev, h->device);
      return PINN_ERR_INVALID_ARG;
    }
  }
  pinn_status s = validate_batch(h, b);
  if (s) return s;
  if (h->spec.ff_m && !h->ff_B) { set_err(h, "Fourier-feature matrix not set (pinn_set_ff_matrix)"); return PINN_ERR_INVALID_ARG; }
  const int64_t N = b->n_res + b->n_ic + b->n_bc;
  *pc = PassCtx{b->n_res, b->n_ic, b->n_bc, true, true, nullptr};
  if (h->global_counts) {
    // a shard of a larger batch: every mean is over the whole batch's points
    if (b->n_res > h->g_res || b->n_ic > h->g_ic || b->n_bc > h->g_bc) {
      set_err(h, "batch has more points than the global counts set by pinn_set_global_counts");
      return PINN_ERR_INVALID_ARG;
    }
    if (h->causal_M > 0) {
      set_err(h, "temporal causality needs every segment's loss, not one shard's");
      return PINN_ERR_UNSUPPORTED;
    }
    pc->N_res = h->g_res; pc->N_ic = h->g_ic; pc->N_bc = h->g_bc;
  }
  if (h->causal_M > 0 && h->chunk_points > 0 && N > h->chunk_points) {
    set_err(h, "temporal causality needs all points in one pass (the weights depend on every segment)");
    return PINN_ERR_UNSUPPORTED;
  }
  return PINN_OK;
}

pinn_status run(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params, void* d_ws,
                size_t ws_bytes, double* d_loss, float* d_grad, void* stream, bool want_grad,
                float* d_grad_terms = nullptr, float* d_grad_ff = nullptr) {
  PassCtx pc;
  pinn_status s = check_call(h, prob, b, d_params, d_ws, d_loss, d_grad, want_grad, d_grad_terms, &pc);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  const int64_t N = b->n_res + b->n_ic + b->n_bc;
  if (h->chunk_points <= 0 || N <= h->chunk_points)
    return run_pass(h, prob, b, d_params, ws, ws_bytes, d_loss, d_grad, st, want_grad, pc, d_grad_terms, d_grad_ff);

  const int64_t C = h->chunk_points;
  const size_t need = chunked_bytes(h, b->n_res, b->n_ic, b->n_bc);
  if (ws_bytes < need) { set_err(h, "workspace too small: %zu < %zu bytes", ws_bytes, need); return PINN_ERR_WORKSPACE; }
  const ChunkLayout cl = chunk_layout(h, C);
  pc.loss_acc = reinterpret_cast<double*>(ws + cl.acc);
  for (int64_t s0 = 0; s0 < N; s0 += C) {
    const int64_t s1 = std::min(N, s0 + C);
    const ChunkRange r = chunk_range(s0, s1, b->n_res, b->n_ic, b->n_bc);
    pinn_batch cb = *b;
    cb.n_res = r.nr; cb.n_ic = r.ni; cb.n_bc = r.nb;
    cb.x_res = reinterpret_cast<float*>(ws + cl.x_res);
    cb.x_ic = reinterpret_cast<float*>(ws + cl.x_ic);
    cb.g_ic = reinterpret_cast<float*>(ws + cl.g_ic);
    cb.x_bc = reinterpret_cast<float*>(ws + cl.x_bc);
    cb.g_bc = reinterpret_cast<float*>(ws + cl.g_bc);
    cudaError_t e = copy_rows(const_cast<float*>(cb.x_res), b->x_res, h->d_in, b->n_res, r.r0, r.nr, st);
    if (e == cudaSuccess) e = copy_rows(const_cast<float*>(cb.x_ic), b->x_ic, h->d_in, b->n_ic, r.i0, r.ni, st);
    if (e == cudaSuccess && b->ic_mask)
      e = copy_rows(const_cast<float*>(cb.g_ic), b->g_ic, h->d_out, b->n_ic, r.i0, r.ni, st);
    if (e == cudaSuccess) e = copy_rows(const_cast<float*>(cb.x_bc), b->x_bc, h->d_in, b->n_bc, r.b0, r.nb, st);
    if (e == cudaSuccess && b->bc_mask)
      e = copy_rows(const_cast<float*>(cb.g_bc), b->g_bc, h->d_out, b->n_bc, r.b0, r.nb, st);
    if (e != cudaSuccess) return cuda_check(h, e, "chunk staging copy");
    pc.first = (s0 == 0);
    pc.last = (s1 == N);
    s = run_pass(h, prob, &cb, d_params, ws + cl.pass, ws_bytes - cl.pass, d_loss, d_grad, st, want_grad, pc,
                 d_grad_terms, d_grad_ff);
    if (s) return s;
  }
  return PINN_OK;
}

// One call by kind: 0 loss, 1 loss+grad, 2 loss+grad+input-map gradient, 3 per-term grads.
pinn_status run_kind(pinn_handle* h, int kind, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                     void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad, float* out2, void* stream) {
  switch (kind) {
    case 0: return run(h, prob, b, d_params, d_ws, ws_bytes, d_loss, nullptr, stream, false);
    case 1: return run(h, prob, b, d_params, d_ws, ws_bytes, d_loss, d_grad, stream, true);
    case 2: return run(h, prob, b, d_params, d_ws, ws_bytes, d_loss, d_grad, stream, true, nullptr, out2);
    default: return run(h, prob, b, d_params, d_ws, ws_bytes, d_loss, nullptr, stream, true, out2);
  }
}

void drop_graph(pinn_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
  memset(&h->graph_key, 0, sizeof(h->graph_key));
}

// run_kind, replayed from a captured CUDA graph when the handle asks for it.
pinn_status run_graphed(pinn_handle* h, int kind, const pinn_problem* prob, const pinn_batch* b,
                        const float* d_params, void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad,
                        float* out2, void* stream) {
  if (!h || !h->graph_on || h->prof || !prob || !b)
    return run_kind(h, kind, prob, b, d_params, d_ws, ws_bytes, d_loss, d_grad, out2, stream);
  pinn_graph_key k;
  memset(&k, 0, sizeof(k));
  k.kind = kind; k.prob = *prob; k.batch = *b;
  k.params = d_params; k.ws = d_ws; k.ws_bytes = ws_bytes; k.loss = d_loss; k.grad = d_grad; k.out2 = out2;
  k.chunk_points = h->chunk_points;
  k.global_counts = h->global_counts ? 1 : 0; k.g_res = h->g_res; k.g_ic = h->g_ic; k.g_bc = h->g_bc;
  k.causal_M = h->causal_M; k.causal_eps = h->causal_eps; k.causal_t0 = h->causal_t0; k.causal_t1 = h->causal_t1;
  k.act = h->act; k.omega0 = h->omega0;
  k.ff_B = h->ff_B; k.periodic = h->periodic ? 1 : 0;
  for (int i = 0; i < 3; ++i) k.periods[i] = h->periods[i];
  k.stream = stream;
  if (!h->graph_exec || memcmp(&k, &h->graph_key, sizeof(k)) != 0) {
    drop_graph(h);
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      set_err(h, "cannot begin stream capture");
      return PINN_ERR_CUDA;
    }
    const pinn_status s = run_kind(h, kind, prob, b, d_params, d_ws, ws_bytes, d_loss, d_grad, out2, h->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (s || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!s) set_err(h, "graph capture failed: %s", cudaGetErrorString(e));
      return s ? s : PINN_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->graph_exec = nullptr;
      return cuda_check(h, ei, "graph instantiation");
    }
    h->graph_key = k;
  }
  return cuda_check(h, cudaGraphLaunch(h->graph_exec, (cudaStream_t)stream), "graph launch");
}

}  // namespace

namespace pinn {

pinn_status loss_grad_eager(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                            void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad, void* stream) {
  return run_kind(h, 1, prob, b, d_params, d_ws, ws_bytes, d_loss, d_grad, nullptr, stream);
}

struct StagedPass {
  Pass pass;
};

pinn_status staged_create(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                          void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad, StagedPass** out) {
  *out = nullptr;
  PassCtx pc;
  pinn_status s = check_call(h, prob, b, d_params, d_ws, d_loss, d_grad, true, nullptr, &pc);
  if (s) return s;
  if (h->chunk_points > 0 && b->n_res + b->n_ic + b->n_bc > h->chunk_points) {
    set_err(h, "a staged pass covers the whole batch in one pass (no point chunking)");
    return PINN_ERR_UNSUPPORTED;
  }
  StagedPass* sp = new (std::nothrow) StagedPass();
  if (!sp) return PINN_ERR_OOM;
  Pass& p = sp->pass;
  p.h = h; p.prob = prob; p.b = b; p.d_params = d_params; p.ws = (char*)d_ws; p.d_loss = d_loss; p.d_grad = d_grad;
  p.want_grad = true; p.pc = pc;
  s = p.init(ws_bytes);
  if (s) { delete sp; return s; }
  *out = sp;
  return PINN_OK;
}

void staged_destroy(StagedPass* sp) { delete sp; }

int staged_forward_levels(const StagedPass* sp) { return sp->pass.h->L - sp->pass.h->first_gemm; }

pinn_status staged_prologue(StagedPass* sp, cudaStream_t st) { return sp->pass.prologue(st); }

pinn_status staged_forward(StagedPass* sp, int level, cudaStream_t st) {
  return sp->pass.forward(sp->pass.h->first_gemm + level, st);
}

pinn_status staged_output(StagedPass* sp, cudaStream_t st) { return sp->pass.output(0, st); }

pinn_status staged_backward(StagedPass* sp, int level, cudaStream_t st) {
  return sp->pass.backward(sp->pass.h->L - 1 - level, st);
}

pinn_status staged_finalize(StagedPass* sp, cudaStream_t st) {
  const pinn_status s = sp->pass.finalize(st);
  return s ? s : cuda_check(sp->pass.h, cudaGetLastError(), "loss_grad launch");
}

}  // namespace pinn

extern "C" {

pinn_status pinn_set_causal(pinn_handle* h, int segments, double eps, double t0, double t1) {
  if (!h || segments < 0 || segments > CAUSAL_MAX || !(eps >= 0.0) || !(t1 > t0)) return PINN_ERR_INVALID_ARG;
  if (segments > 0 && h->spec.pde == PINN_NS_STEADY_2D) {
    set_err(h, "the steady Navier-Stokes problem has no time input");
    return PINN_ERR_UNSUPPORTED;
  }
  h->causal_M = segments;
  h->causal_eps = eps;
  h->causal_t0 = t0;
  h->causal_t1 = t1;
  return PINN_OK;
}

pinn_status pinn_causal_weights(pinn_handle* h, double* d_weights, void* stream) {
  if (!h || !d_weights || h->causal_M <= 0) return PINN_ERR_INVALID_ARG;
  return cuda_check(h, cudaMemcpyAsync(d_weights, h->d_scratch + 256, sizeof(double) * h->causal_M,
                                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                    "causal weights copy");
}

pinn_status pinn_set_chunk_points(pinn_handle* h, int64_t points) {
  if (!h || points < 0) return PINN_ERR_INVALID_ARG;
  h->chunk_points = (int64_t)align_up((size_t)points, PT_ALIGN);
  return PINN_OK;
}

pinn_status pinn_set_global_counts(pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc) {
  if (!h || n_res < 0 || n_ic < 0 || n_bc < 0) return PINN_ERR_INVALID_ARG;
  h->global_counts = (n_res + n_ic + n_bc) > 0;
  h->g_res = n_res; h->g_ic = n_ic; h->g_bc = n_bc;
  return PINN_OK;
}

pinn_status pinn_set_graph(pinn_handle* h, int on) {
  if (!h || (on != 0 && on != 1)) return PINN_ERR_INVALID_ARG;
  if (on && !h->cap_stream) {
    pinn_status s = cuda_check(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (s) return s;
  }
  if (!on) drop_graph(h);
  h->graph_on = on != 0;
  return PINN_OK;
}

pinn_status pinn_graph_held(const pinn_handle* h, int32_t* held) {
  if (!h || !held) return PINN_ERR_INVALID_ARG;
  *held = h->graph_exec ? 1 : 0;
  return PINN_OK;
}

pinn_status pinn_set_activation(pinn_handle* h, int act, double omega0) {
  if (!h) return PINN_ERR_INVALID_ARG;
  if (act != PINN_ACT_TANH && act != PINN_ACT_SINE) { set_err(h, "unknown activation %d", act); return PINN_ERR_INVALID_ARG; }
  if (!(omega0 > 0.0) || !std::isfinite(omega0) || omega0 > 1e4) {
    set_err(h, "omega0 must be finite and in (0, 1e4]"); return PINN_ERR_INVALID_ARG;
  }
  h->act = act;
  h->omega0 = (float)omega0;
  return PINN_OK;
}

pinn_status pinn_create(const pinn_spec* spec, pinn_handle** out) {
  if (!spec || !out) return PINN_ERR_INVALID_ARG;
  *out = nullptr;
  if (spec->pde < 0 || spec->pde > PINN_ALLEN_CAHN_1D) return PINN_ERR_INVALID_ARG;
  if (spec->n_hidden < 1 || spec->n_hidden > PINN_MAX_HIDDEN) return PINN_ERR_INVALID_ARG;
  for (int i = 0; i < spec->n_hidden; ++i)
    if (spec->widths[i] < 1 || spec->widths[i] > 2048) return PINN_ERR_INVALID_ARG;
  if (spec->ff_m < 0 || spec->ff_m > 2048) return PINN_ERR_INVALID_ARG;
  if (spec->rwf != 0 && spec->rwf != 1) return PINN_ERR_INVALID_ARG;
  if (spec->precision < PINN_FP32 || spec->precision > PINN_BF16) return PINN_ERR_INVALID_ARG;
  if (spec->flags & ~(PINN_FLAG_CUDA_CORES | PINN_FLAG_BF16_VALUE_SPLIT | PINN_FLAG_UNFUSED_ADJOINT |
                      PINN_FLAG_DW_ROWS_128))
    return PINN_ERR_INVALID_ARG;
  pinn_handle* h = new (std::nothrow) pinn_handle();
  if (!h) return PINN_ERR_OOM;
  h->spec = *spec;
  h->L = spec->n_hidden;
  h->d_in = pde_din(spec->pde);
  h->d_out = pde_dout(spec->pde);
  // scalar 1-D problems carry [u, u_x, u_t, u_xx]
  h->jet_mode = spec->pde == PINN_NS_STEADY_2D ? JET_NS : spec->pde == PINN_MAXWELL_TE_2D ? JET_MAXWELL : JET_BURGERS;
  h->first_gemm = spec->ff_m ? 0 : 1;
  int64_t off = 0;
  int prev = spec->ff_m ? 2 * spec->ff_m : h->d_in;
  h->w_max = 0;
  for (int li = 0; li <= h->L; ++li) {
    const int fout = li < h->L ? spec->widths[li] : h->d_out;
    LayerPlan& lp = h->layers[li];
    lp.fin = prev; lp.fout = fout;
    lp.off_V = off; off += (int64_t)prev * fout;
    if (spec->rwf) { lp.off_s = off; off += fout; } else lp.off_s = -1;
    lp.off_b = off; off += fout;
    if (li < h->L) h->w_max = std::max(h->w_max, fout);
    prev = fout;
  }
  h->P = off;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, 256);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_scratch, 4096);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->d_status) cudaFree(h->d_status);
    if (h->d_scratch) cudaFree(h->d_scratch);
    delete h;
    return e == cudaErrorMemoryAllocation ? PINN_ERR_OOM : PINN_ERR_CUDA;
  }
  tc_init(h);
  *out = h;
  return PINN_OK;
}

pinn_status pinn_destroy(pinn_handle* h) {
  if (!h) return PINN_OK;
  if (h->prof_ev) {
    for (int i = 0; i < 2 * PROF_MAX; ++i) cudaEventDestroy(h->prof_ev[i]);
    delete[] h->prof_ev;
    delete[] h->prof_phase;
    delete[] h->prof_launches;
  }
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_scratch) cudaFree(h->d_scratch);
  if (h->d_periodic_B) cudaFree(h->d_periodic_B);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return PINN_OK;
}

pinn_status pinn_param_count(const pinn_handle* h, int64_t* P) {
  if (!h || !P) return PINN_ERR_INVALID_ARG;
  *P = h->P;
  return PINN_OK;
}

pinn_status pinn_workspace_bytes(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, size_t* bytes) {
  if (!h || !bytes || n_res < 0 || n_ic < 0 || n_bc < 0) return PINN_ERR_INVALID_ARG;
  const int64_t N = n_res + n_ic + n_bc;
  if (h->chunk_points > 0 && N > h->chunk_points) {
    *bytes = chunked_bytes(h, n_res, n_ic, n_bc);
    return PINN_OK;
  }
  CallPlan cp;
  plan_call(h, n_res, n_ic, n_bc, &cp);
  *bytes = cp.p.total;
  return PINN_OK;
}

pinn_status pinn_tensor_core_layers(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, int32_t* n) {
  if (!h || !n || n_res < 0 || n_ic < 0 || n_bc < 0) return PINN_ERR_INVALID_ARG;
  CallPlan cp;
  plan_call(h, n_res, n_ic, n_bc, &cp);
  int32_t c = 0;
  for (int li = 0; li < h->L; ++li) c += cp.tc[li] ? 1 : 0;
  *n = c;
  return PINN_OK;
}

pinn_status pinn_layer_engines(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, int32_t* engines) {
  if (!h || !engines || n_res < 0 || n_ic < 0 || n_bc < 0) return PINN_ERR_INVALID_ARG;
  CallPlan cp;
  plan_call(h, n_res, n_ic, n_bc, &cp);
  for (int li = 0; li < h->L; ++li) engines[li] = cp.fused[li] ? 2 : cp.tc[li] ? 1 : 0;
  return PINN_OK;
}

pinn_status pinn_set_ff_matrix(pinn_handle* h, const float* d_B) {
  if (!h || !d_B) return PINN_ERR_INVALID_ARG;
  if (!h->spec.ff_m) { set_err(h, "network has no Fourier features"); return PINN_ERR_INVALID_ARG; }
  h->ff_B = d_B;
  h->periodic = false;
  return PINN_OK;
}

pinn_status pinn_set_periodic(pinn_handle* h, const double* periods) {
  if (!h || !periods) return PINN_ERR_INVALID_ARG;
  if (h->spec.ff_m != h->d_in) {
    set_err(h, "the periodic input map needs ff_m = d_in (%d), got %d", h->d_in, h->spec.ff_m);
    return PINN_ERR_INVALID_ARG;
  }
  for (int k = 0; k < h->d_in; ++k)
    if (!(periods[k] > 0.0) || !std::isfinite(periods[k])) { set_err(h, "periods must be finite and > 0"); return PINN_ERR_INVALID_ARG; }
  const int d = h->d_in;
  if (!h->d_periodic_B) {
    const cudaError_t e = cudaMalloc(&h->d_periodic_B, (size_t)d * d * sizeof(float));
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); set_err(h, "periodic map alloc: out of memory"); return PINN_ERR_OOM; }
    pinn_status s = cuda_check(h, e, "periodic map alloc");
    if (s) return s;
  }
  float Bh[9] = {0.f};
  for (int k = 0; k < d; ++k) Bh[k * d + k] = (float)(2.0 * 3.14159265358979323846 / periods[k]);
  pinn_status s = cuda_check(h, cudaMemcpy(h->d_periodic_B, Bh, (size_t)d * d * sizeof(float), cudaMemcpyHostToDevice),
                             "periodic map upload");
  if (s) return s;
  for (int k = 0; k < d; ++k) h->periods[k] = periods[k];
  h->ff_B = h->d_periodic_B;
  h->periodic = true;
  return PINN_OK;
}

pinn_status pinn_loss_grad_ff(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch, const float* d_params,
                              void* d_ws, size_t ws_bytes, double* d_loss_terms, float* d_grad, float* d_grad_ff,
                              void* stream) {
  if (!h) return PINN_ERR_INVALID_ARG;
  if (!h->spec.ff_m) { set_err(h, "network has no input map (Fourier features or periodic)"); return PINN_ERR_INVALID_ARG; }
  if (!d_grad_ff) { set_err(h, "NULL argument"); return PINN_ERR_INVALID_ARG; }
  return run_graphed(h, 2, prob, batch, d_params, d_ws, ws_bytes, d_loss_terms, d_grad, d_grad_ff, stream);
}

pinn_status pinn_loss(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch, const float* d_params,
                      void* d_ws, size_t ws_bytes, double* d_loss_terms, void* stream) {
  return run_graphed(h, 0, prob, batch, d_params, d_ws, ws_bytes, d_loss_terms, nullptr, nullptr, stream);
}

pinn_status pinn_loss_grad_terms(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                                 const float* d_params, void* d_ws, size_t ws_bytes, double* d_loss_terms,
                                 float* d_grad_terms, void* stream) {
  if (!d_grad_terms) { if (h) set_err(h, "NULL argument"); return PINN_ERR_INVALID_ARG; }
  return run_graphed(h, 3, prob, batch, d_params, d_ws, ws_bytes, d_loss_terms, nullptr, d_grad_terms, stream);
}

pinn_status pinn_loss_balance(pinn_handle* h, const float* d_grad_terms, double* d_lambda, double* d_norms,
                              double alpha, double eps, int update, void* stream) {
  if (!h || !d_grad_terms || !d_lambda || !(alpha >= 0.0 && alpha <= 1.0) || !(eps >= 0.0))
    return PINN_ERR_INVALID_ARG;
  launch_loss_balance(d_grad_terms, h->P, d_lambda, d_norms, alpha, eps, update, h->d_scratch, (cudaStream_t)stream);
  return cuda_check(h, cudaGetLastError(), "loss-balance launch");
}

pinn_status pinn_loss_grad(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch, const float* d_params,
                           void* d_ws, size_t ws_bytes, double* d_loss_terms, float* d_grad, void* stream) {
  return run_graphed(h, 1, prob, batch, d_params, d_ws, ws_bytes, d_loss_terms, d_grad, nullptr, stream);
}

pinn_status pinn_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t n, int64_t step,
                           float lr, float beta1, float beta2, float eps, void* stream) {
  if (!d_params || !d_grad || !d_m || !d_v || n < 0 || step < 1) return PINN_ERR_INVALID_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return PINN_ERR_INVALID_ARG;
  if (n == 0) return PINN_OK;
  const double bc1 = 1.0 - std::pow((double)beta1, (double)step);
  const double bc2 = 1.0 - std::pow((double)beta2, (double)step);
  launch_adam(d_params, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, (float)bc1, (float)bc2, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}

pinn_status pinn_status_poll(pinn_handle* h, void* stream) {
  if (!h) return PINN_ERR_INVALID_ARG;
  pinn_status s = cuda_check(h, cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
  if (s) return s;
  int v = 0;
  s = cuda_check(h, cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (s) return s;
  if (v) cudaMemset(h->d_status, 0, sizeof(int));
  if (v & 2) { set_err(h, "a device-side wait exceeded its bound"); return PINN_ERR_TIMEOUT; }
  if (v & 1) { set_err(h, "non-finite loss"); return PINN_ERR_NONFINITE; }
  return PINN_OK;
}

pinn_status pinn_set_profiling(pinn_handle* h, int enable) {
  if (!h) return PINN_ERR_INVALID_ARG;
  if (enable && !h->prof_ev) {
    h->prof_ev = new (std::nothrow) cudaEvent_t[2 * PROF_MAX];
    h->prof_phase = new (std::nothrow) int[PROF_MAX];
    h->prof_launches = new (std::nothrow) int[PROF_MAX];
    if (!h->prof_ev || !h->prof_phase || !h->prof_launches) return PINN_ERR_INVALID_ARG;
    for (int i = 0; i < 2 * PROF_MAX; ++i) {
      pinn_status s = cuda_check(h, cudaEventCreate(&h->prof_ev[i]), "profiler event");
      if (s) return s;
    }
  }
  h->prof = enable != 0;
  h->prof_n = 0;
  h->prof_dropped = 0;
  return PINN_OK;
}

pinn_status pinn_profile_read(pinn_handle* h, double* ms, int64_t* launches) {
  if (!h || !ms || !launches) return PINN_ERR_INVALID_ARG;
  for (int i = 0; i < PINN_PROF_PHASES; ++i) { ms[i] = 0.0; launches[i] = 0; }
  if (h->prof_n > 0) {
    pinn_status s = cuda_check(h, cudaEventSynchronize(h->prof_ev[2 * h->prof_n - 1]), "profiler sync");
    if (s) return s;
    for (int i = 0; i < h->prof_n; ++i) {
      float t = 0.f;
      s = cuda_check(h, cudaEventElapsedTime(&t, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]), "profiler elapsed");
      if (s) return s;
      ms[h->prof_phase[i]] += t;
      launches[h->prof_phase[i]] += h->prof_launches[i];
    }
  }
  if (h->prof_dropped) launches[PINN_PROF_PHASES - 1] = -1;
  h->prof_n = 0;
  h->prof_dropped = 0;
  return PINN_OK;
}

const char* pinn_last_error(const pinn_handle* h) { return h ? h->err : "NULL handle"; }

const char* pinn_status_string(pinn_status s) {
  switch (s) {
    case PINN_OK: return "PINN_OK";
    case PINN_ERR_INVALID_ARG: return "PINN_ERR_INVALID_ARG";
    case PINN_ERR_UNSUPPORTED: return "PINN_ERR_UNSUPPORTED";
    case PINN_ERR_CUDA: return "PINN_ERR_CUDA";
    case PINN_ERR_WORKSPACE: return "PINN_ERR_WORKSPACE";
    case PINN_ERR_NONFINITE: return "PINN_ERR_NONFINITE";
    case PINN_ERR_TIMEOUT: return "PINN_ERR_TIMEOUT";
    case PINN_ERR_OOM: return "PINN_ERR_OOM";
  }
  return "PINN_ERR_UNKNOWN";
}

const char* pinn_version(void) { return "pinn-gb300 0.1 (sm_103a)"; }

}  // extern "C"
