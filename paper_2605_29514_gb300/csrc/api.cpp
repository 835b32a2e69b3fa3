// C ABI of the simulator (declared in include/stn.h): context, device memory
// plan, batch control and result readback.  All launches go to the stream the
// context was created with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/stn.h"
#include "engine.h"
#include "program.h"

struct stn_ctx {
  stn_config cfg{};
  stn::Program prog;
  cudaStream_t stream = nullptr;
  int64_t max_shots = 0, shots = 0;
  uint64_t shot_offset = 0;
  int n = 0, W = 0, rec_bytes = 0, K = 0, grid = 1, svd_elems = 0;
  std::vector<int> chimax;
  std::vector<int64_t> site_off;
  int64_t slab_elems = 0;
  size_t elem = 8;
  stn::ScratchPlan plan{};
  // device memory
  stn::Op *d_ops = nullptr;
  double *d_theta = nullptr;
  uint64_t *d_tx = nullptr, *d_tz = nullptr;
  uint8_t *d_tm = nullptr;
  void *d_mps = nullptr;
  int64_t *d_site_off = nullptr;
  int *d_chimax = nullptr;
  int *d_chi = nullptr, *d_center = nullptr, *d_maxchi = nullptr, *d_near = nullptr,
      *d_status = nullptr;
  double *d_logp = nullptr, *d_disc = nullptr, *d_born = nullptr, *d_flops = nullptr;
  double *d_prof = nullptr;
  uint8_t *d_rec = nullptr, *d_det = nullptr, *d_obs = nullptr;
  int32_t *d_det_table = nullptr, *d_logical = nullptr;
  void *d_scratch = nullptr;
  int *d_err = nullptr;
  uint64_t *d_offset = nullptr;  // shot offset read by captured graphs
  int *d_ticket = nullptr;       // shot queue of a round-kernel launch
  cudaGraphExec_t graph = nullptr;
  int64_t graph_shots = 0;
  double *d_diag = nullptr;     // diagnostics output: max(max_shots, 512) doubles
  int *d_diag_count = nullptr;
  int32_t *d_diag_q = nullptr;  // n qubit indices
  std::string last_error;
  std::vector<void *> allocs;
};

namespace {

stn_status fail(stn_ctx *c, stn_status st, const std::string &msg) {
  if (c) c->last_error = msg;
  return st;
}

stn_status cuda_fail(stn_ctx *c, cudaError_t e, const char *where) {
  return fail(c, STN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename P>
cudaError_t dalloc(stn_ctx *c, P **ptr, size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    c->allocs.push_back(p);
    *ptr = static_cast<P *>(p);
  }
  return e;
}

stn::EngineParams params(const stn_ctx *c, int op_begin, int op_end, const double *d_theta) {
  stn::EngineParams p{};
  p.ops = c->d_ops;
  p.op_begin = op_begin;
  p.op_end = op_end;
  p.theta = d_theta;
  p.n = c->n;
  p.W = c->W;
  p.n_meas = c->prog.n_meas;
  p.rec_bytes = c->rec_bytes;
  p.chi_cap = c->cfg.chi_cap;
  p.cutoff = c->cfg.svd_cutoff;
  p.delta = c->cfg.degeneracy_tol;
  p.p1 = c->cfg.p * c->cfg.p1_scale;
  p.p2 = c->cfg.p * c->cfg.p2_scale;
  p.pR = c->cfg.p * c->cfg.pR_scale;
  p.pM = c->cfg.p * c->cfg.pM_scale;
  p.seed = c->cfg.seed;
  p.shot_offset = c->shot_offset;
  p.shots = static_cast<int>(c->shots);
  p.tab_x = c->d_tx;
  p.tab_z = c->d_tz;
  p.tab_m = c->d_tm;
  p.mps = c->d_mps;
  p.site_off = c->d_site_off;
  p.chimax = c->d_chimax;
  p.slab_elems = c->slab_elems;
  p.chi = c->d_chi;
  p.center = c->d_center;
  p.logp = c->d_logp;
  p.disc = c->d_disc;
  p.maxchi = c->d_maxchi;
  p.near = c->d_near;
  p.status = c->d_status;
  p.records = c->d_rec;
  p.born = c->d_born;
  p.flops = c->d_flops;
  p.prof = c->d_prof;
  p.scratch = c->d_scratch;
  p.scratch_elems = c->plan.total;
  p.ap_elems = c->plan.ap_elems;
  p.g_elems = c->plan.g_elems;
  p.work_c = c->plan.work_c;
  p.svd_elems = c->svd_elems;
  p.svd64_all = c->cfg.precision == STN_PRECISION_C64_SVD64 ? 1 : 0;
  p.use_tc = c->cfg.precision != STN_PRECISION_C128 && c->cfg.gemm_units == STN_GEMM_TENSOR ? 1 : 0;
  p.err = c->d_err;
  return p;
}

std::string validate(const stn_config *cfg) {
  if (!cfg) return "config is NULL";
  if (cfg->chi_cap < 1 || cfg->chi_cap > 256) return "chi_cap must be 1..256";
  if (cfg->precision != STN_PRECISION_C128 && cfg->precision != STN_PRECISION_C64 &&
      cfg->precision != STN_PRECISION_C64_SVD64)
    return "precision must be one of STN_PRECISION_*";
  const double rates[5] = {cfg->p, cfg->p1_scale, cfg->p2_scale, cfg->pR_scale, cfg->pM_scale};
  for (double r : rates)
    if (!(r >= 0.0) || !std::isfinite(r)) return "noise rates must be finite and >= 0";
  const double probs[4] = {cfg->p * cfg->p1_scale, cfg->p * cfg->p2_scale, cfg->p * cfg->pR_scale,
                           cfg->p * cfg->pM_scale};
  for (double r : probs)
    if (r > 1.0) return "scaled noise probabilities must be <= 1";
  if (!(cfg->svd_cutoff >= 0.0) || !(cfg->svd_cutoff < 1.0)) return "svd_cutoff must be in [0, 1)";
  if (!(cfg->degeneracy_tol >= 0.0) || !(cfg->degeneracy_tol < 1.0))
    return "degeneracy_tol must be in [0, 1)";
  if (cfg->distance > 9) return "distance must be <= 9";
  if (cfg->memory_basis != STN_BASIS_Z && cfg->memory_basis != STN_BASIS_X)
    return "memory_basis must be STN_BASIS_Z or STN_BASIS_X";
  if (cfg->n_pairs < 0 || cfg->n_pairs > 4096) return "n_pairs must be 0..4096";
  if (cfg->n_pairs > 0 && !cfg->pairs) return "pairs is NULL with n_pairs > 0";
  if (cfg->arena_cap_bytes < 0) return "arena_cap_bytes must be >= 0";
  if (cfg->gemm_units != STN_GEMM_TENSOR && cfg->gemm_units != STN_GEMM_FMA)
    return "gemm_units must be STN_GEMM_TENSOR or STN_GEMM_FMA";
  return std::string();
}

// The program spec of a validated config, with the caller's arrays copied.
std::string make_spec(const stn_config *cfg, stn::ProgramSpec &sp) {
  std::string why = validate(cfg);
  if (!why.empty()) return why;
  sp = stn::ProgramSpec();
  sp.d = cfg->distance;
  sp.rounds = cfg->rounds;
  sp.pair_rule = cfg->pair_rule;
  sp.basis = cfg->memory_basis;
  if (cfg->cnot_schedule) {
    const int n_anc = cfg->distance * cfg->distance - 1;
    sp.schedule.assign(cfg->cnot_schedule, cfg->cnot_schedule + 4 * n_anc);
  }
  if (cfg->n_pairs > 0) {
    sp.explicit_pairs = true;
    for (int k = 0; k < cfg->n_pairs; ++k) {
      stn::Pair p{};
      p.a = cfg->pairs[2 * k];
      p.b = cfg->pairs[2 * k + 1];
      p.pauli = cfg->pair_pauli ? cfg->pair_pauli[k] : 0;
      const int lm = cfg->pair_layer_mask ? cfg->pair_layer_mask[k] : STN_LAYERS_IDLE;
      p.layer_mask = lm == STN_LAYERS_IDLE ? -1 : (lm & 0xF);
      sp.pairs.push_back(p);
    }
  }
  return std::string();
}

std::string compile(const stn_config *cfg, stn::Program &prog) {
  stn::ProgramSpec sp;
  std::string why = make_spec(cfg, sp);
  if (!why.empty()) return why;
  return stn::build_program(sp, prog);
}

}  // namespace

namespace {
// Device buffers of one adjoint call, freed when it returns.
struct AdjointBuffers {
  std::vector<void *> ptrs;
  ~AdjointBuffers() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename P>
  bool get(P **out, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ptrs.push_back(p);
    *out = static_cast<P *>(p);
    return true;
  }
};
}  // namespace

extern "C" {

int32_t stn_layout(int32_t distance, int32_t *h_xy, char *h_kind) {
  stn::ProgramSpec sp;
  sp.d = distance;
  sp.rounds = 1;
  stn::Program prog;
  if (!stn::build_program(sp, prog).empty()) return -1;
  for (int q = 0; q < prog.n; ++q) {
    if (h_xy) {
      h_xy[2 * q] = prog.xy[2 * q];
      h_xy[2 * q + 1] = prog.xy[2 * q + 1];
    }
    if (h_kind) h_kind[q] = prog.kind[q];
  }
  return prog.n;
}

stn_status stn_create(const stn_config *cfg, int64_t max_shots, void *cuda_stream, stn_ctx **out) {
  if (!out) return STN_EINVAL;
  *out = nullptr;
  std::string why = validate(cfg);
  if (!why.empty()) return STN_EINVAL;
  if (max_shots < 1 || max_shots > (1ll << 31)) return STN_EINVAL;
  stn_ctx *c = new (std::nothrow) stn_ctx();
  if (!c) return STN_ENOMEM;
  c->cfg = *cfg;
  // the arrays were copied into the program; the context keeps no caller pointer
  c->cfg.cnot_schedule = nullptr;
  c->cfg.pairs = nullptr;
  c->cfg.pair_pauli = nullptr;
  c->cfg.pair_layer_mask = nullptr;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->max_shots = max_shots;
  why = compile(cfg, c->prog);
  if (!why.empty()) {
    delete c;
    return STN_EINVAL;
  }
  const int n = c->n = c->prog.n;
  c->W = (n + 63) / 64;
  c->rec_bytes = (c->prog.n_meas + 7) / 8;
  c->K = static_cast<int>(c->prog.pairs.size());
  c->elem = cfg->precision == STN_PRECISION_C128 ? 16 : 8;
  // largest bond per cut: the cap, and 2^min(k, n-k) (Schmidt rank bound)
  c->chimax.assign(n + 1, 1);
  for (int k = 1; k < n; ++k) {
    int e = std::min(k, n - k);
    int64_t v = e >= 30 ? (1ll << 30) : (1ll << e);
    c->chimax[k] = static_cast<int>(std::min<int64_t>(v, cfg->chi_cap));
  }
  c->site_off.assign(n + 1, 0);
  for (int k = 0; k < n; ++k)
    c->site_off[k + 1] = c->site_off[k] + 2ll * c->chimax[k] * c->chimax[k + 1];
  c->slab_elems = c->site_off[n];
  c->plan = stn::plan_scratch(n, c->chimax.data(), cfg->chi_cap);
  if (cfg->arena_cap_bytes > 0) {  // shrink the span stacks to the caller's cap
    const int64_t cap = cfg->arena_cap_bytes / static_cast<int64_t>(c->elem);
    const int64_t need = c->plan.ap_elems + c->plan.g_elems;
    if (cap < need) {
      const double f = static_cast<double>(cap) / static_cast<double>(need);
      c->plan.ap_elems = static_cast<int64_t>(static_cast<double>(c->plan.ap_elems) * f);
      c->plan.g_elems = static_cast<int64_t>(static_cast<double>(c->plan.g_elems) * f);
      c->plan.total = c->plan.ap_elems + c->plan.g_elems + c->plan.work_elems;
    }
  }
  c->svd_elems = stn::round_kernel_svd_elems(cfg->precision, n, c->W);
  if (c->svd_elems < 2 * 4 * c->plan.work_c + 16) {  // the blocked SVD needs two columns
    delete c;
    return STN_EINVAL;
  }

  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return STN_ECUDA;
  }
  c->grid = static_cast<int>(std::min<int64_t>(max_shots, sms));

  const int64_t S = max_shots;
  const size_t nn = static_cast<size_t>(2 * n);
  bool ok = true;
  auto A = [&](cudaError_t r) { ok = ok && r == cudaSuccess; };
  A(dalloc(c, &c->d_ops, sizeof(stn::Op) * c->prog.ops.size()));
  A(dalloc(c, &c->d_theta, sizeof(double) * std::max(1, c->K)));
  A(dalloc(c, &c->d_tx, sizeof(uint64_t) * S * nn * c->W));
  A(dalloc(c, &c->d_tz, sizeof(uint64_t) * S * nn * c->W));
  A(dalloc(c, &c->d_tm, S * nn));
  A(dalloc(c, &c->d_mps, c->elem * S * c->slab_elems));
  A(dalloc(c, &c->d_site_off, sizeof(int64_t) * (n + 1)));
  A(dalloc(c, &c->d_chimax, sizeof(int) * (n + 1)));
  A(dalloc(c, &c->d_chi, sizeof(int) * S * (n + 1)));
  A(dalloc(c, &c->d_center, sizeof(int) * S));
  A(dalloc(c, &c->d_maxchi, sizeof(int) * S));
  A(dalloc(c, &c->d_near, sizeof(int) * S));
  A(dalloc(c, &c->d_status, sizeof(int) * S));
  A(dalloc(c, &c->d_logp, sizeof(double) * S));
  A(dalloc(c, &c->d_disc, sizeof(double) * S));
  A(dalloc(c, &c->d_born, sizeof(double) * S * c->prog.n_meas));
  A(dalloc(c, &c->d_flops, sizeof(double) * S));
  A(dalloc(c, &c->d_prof, sizeof(double) * S * stn::kProfSlots));
  A(dalloc(c, &c->d_rec, static_cast<size_t>(S) * c->rec_bytes));
  A(dalloc(c, &c->d_det, static_cast<size_t>(S) * ((c->prog.n_det + 7) / 8)));
  A(dalloc(c, &c->d_obs, static_cast<size_t>(S)));
  A(dalloc(c, &c->d_det_table, sizeof(int32_t) * c->prog.det.size()));
  A(dalloc(c, &c->d_logical, sizeof(int32_t) * c->prog.logical.size()));
  A(dalloc(c, &c->d_scratch, c->elem * static_cast<size_t>(c->grid) * c->plan.total));
  A(dalloc(c, &c->d_err, sizeof(int)));
  A(dalloc(c, &c->d_offset, sizeof(uint64_t)));
  A(dalloc(c, &c->d_ticket, sizeof(int)));
  A(dalloc(c, &c->d_diag, sizeof(double) * std::max<int64_t>(S, 512)));
  A(dalloc(c, &c->d_diag_count, sizeof(int)));
  A(dalloc(c, &c->d_diag_q, sizeof(int32_t) * n));
  if (!ok) {
    stn_destroy(c);
    cudaGetLastError();
    return STN_ENOMEM;
  }
  e = cudaMemcpyAsync(c->d_ops, c->prog.ops.data(), sizeof(stn::Op) * c->prog.ops.size(),
                      cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_site_off, c->site_off.data(), sizeof(int64_t) * (n + 1),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_chimax, c->chimax.data(), sizeof(int) * (n + 1),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_det_table, c->prog.det.data(), sizeof(int32_t) * c->prog.det.size(),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_logical, c->prog.logical.data(), sizeof(int32_t) * c->prog.logical.size(),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flops, 0, sizeof(double) * S, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_prof, 0, sizeof(double) * S * stn::kProfSlots, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    stn_destroy(c);
    return STN_ECUDA;
  }
  *out = c;
  return STN_OK;
}

void stn_destroy(stn_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

const char *stn_last_error(const stn_ctx *c) { return c ? c->last_error.c_str() : "no context"; }

int32_t stn_num_qubits(const stn_ctx *c) { return c ? c->n : -1; }
int32_t stn_num_pairs(const stn_ctx *c) { return c ? c->K : -1; }
int32_t stn_num_meas(const stn_ctx *c) { return c ? c->prog.n_meas : -1; }
int32_t stn_num_events(const stn_ctx *c) { return c ? c->prog.n_events : -1; }
int32_t stn_num_ops(const stn_ctx *c) { return c ? static_cast<int32_t>(c->prog.ops.size()) : -1; }

static void dump_program(const stn::Program &prog, int32_t *h_ops, int32_t *h_pairs) {
  if (h_ops) {
    for (size_t i = 0; i < prog.ops.size(); ++i) {
      const stn::Op &o = prog.ops[i];
      int32_t *r = h_ops + 6 * i;
      r[0] = o.kind; r[1] = o.a; r[2] = o.b; r[3] = o.pauli; r[4] = o.ev; r[5] = o.idx;
    }
  }
  if (h_pairs) {
    for (size_t k = 0; k < prog.pairs.size(); ++k) {
      const stn::Pair &p = prog.pairs[k];
      int32_t *r = h_pairs + 4 * k;
      r[0] = p.a; r[1] = p.b; r[2] = p.pauli; r[3] = p.layer_mask;
    }
  }
}

stn_status stn_get_program(const stn_ctx *c, int32_t *h_ops, int32_t *h_pairs) {
  if (!c) return STN_EINVAL;
  dump_program(c->prog, h_ops, h_pairs);
  return STN_OK;
}

stn_status stn_compile_program(const stn_config *cfg, int32_t *h_counts, int32_t *h_ops,
                               int32_t *h_pairs) {
  stn::Program prog;
  if (!compile(cfg, prog).empty()) return STN_EINVAL;
  if (h_counts) {
    h_counts[0] = prog.n;
    h_counts[1] = static_cast<int32_t>(prog.pairs.size());
    h_counts[2] = prog.n_meas;
    h_counts[3] = prog.n_events;
    h_counts[4] = static_cast<int32_t>(prog.ops.size());
  }
  dump_program(prog, h_ops, h_pairs);
  return STN_OK;
}

stn_status stn_compile_detectors(const stn_config *cfg, int32_t *h_counts, int32_t *h_det,
                                 int32_t *h_logical) {
  stn::Program prog;
  if (!compile(cfg, prog).empty()) return STN_EINVAL;
  if (h_counts) {
    h_counts[0] = prog.n_det;
    h_counts[1] = static_cast<int32_t>(prog.logical.size());
  }
  if (h_det) std::copy(prog.det.begin(), prog.det.end(), h_det);
  if (h_logical) std::copy(prog.logical.begin(), prog.logical.end(), h_logical);
  return STN_OK;
}

stn_status stn_begin_batch(stn_ctx *c, int64_t shots, uint64_t shot_offset) {
  if (!c) return STN_EINVAL;
  if (shots < 1 || shots > c->max_shots) return fail(c, STN_EINVAL, "shots must be 1..max_shots");
  c->shots = shots;
  c->shot_offset = shot_offset;
  cudaError_t e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_begin_batch");
  stn::EngineParams p = params(c, 0, 0, c->d_theta);
  e = stn::launch_init(c->cfg.precision, p, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  return STN_OK;
}

static stn_status launch_ops(stn_ctx *c, int op_begin, int op_end, const double *d_theta) {
  if (c->shots < 1) return fail(c, STN_EINVAL, "no batch: call stn_begin_batch first");
  if (!d_theta && c->K > 0) return fail(c, STN_EINVAL, "theta is NULL");
  stn::EngineParams p = params(c, op_begin, op_end, d_theta ? d_theta : c->d_theta);
  int grid = static_cast<int>(std::min<int64_t>(c->grid, c->shots));
  cudaError_t e = cudaSuccess;
  if (c->shots > grid) {  // more shots than CTAs: take them from a queue
    e = cudaMemsetAsync(c->d_ticket, 0, sizeof(int), c->stream);
    p.ticket = c->d_ticket;
  }
  if (e == cudaSuccess) e = stn::launch_round(c->cfg.precision, p, grid, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "round kernel");
  return STN_OK;
}

stn_status stn_apply_round_device(stn_ctx *c, int32_t round, const double *d_theta) {
  if (!c) return STN_EINVAL;
  if (round < 0 || round > c->cfg.rounds) return fail(c, STN_EINVAL, "round must be 0..rounds");
  return launch_ops(c, c->prog.seg_begin[round], c->prog.seg_begin[round + 1], d_theta);
}

int32_t stn_num_steps(const stn_ctx *c) { return c ? static_cast<int32_t>(c->prog.step_begin.size()) - 1 : -1; }

stn_status stn_apply_step_device(stn_ctx *c, int32_t step, const double *d_theta) {
  if (!c) return STN_EINVAL;
  if (step < 0 || step >= stn_num_steps(c)) return fail(c, STN_EINVAL, "step must be 0..4 rounds - 1");
  return launch_ops(c, c->prog.step_begin[step], c->prog.step_begin[step + 1], d_theta);
}

stn_status stn_apply_round(stn_ctx *c, int32_t round, const double *h_theta) {
  if (!c) return STN_EINVAL;
  if (!h_theta && c->K > 0) return fail(c, STN_EINVAL, "theta is NULL");
  for (int k = 0; k < c->K; ++k)
    if (!std::isfinite(h_theta[k])) return fail(c, STN_EINVAL, "theta must be finite");
  if (c->K > 0) {
    cudaError_t e = cudaMemcpyAsync(c->d_theta, h_theta, sizeof(double) * c->K,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "theta copy");
  }
  return stn_apply_round_device(c, round, c->d_theta);
}

stn_status stn_sync(stn_ctx *c) {
  if (!c) return STN_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream");
  int err = 0;
  e = cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error flag");
  if (err == STN_ENUMERIC) return fail(c, STN_ENUMERIC, "non-finite or vanishing MPS norm in a shot");
  if (err == STN_EOVERFLOW) return fail(c, STN_EOVERFLOW, "scratch arena too small for a sweep");
  if (err != 0) return fail(c, static_cast<stn_status>(err), "device reported an error");
  return STN_OK;
}

stn_status stn_read_records(stn_ctx *c, uint8_t *h_records, double *h_born,
                            stn_shot_stats *h_stats) {
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  cudaError_t e = cudaSuccess;
  if (h_records)
    e = cudaMemcpy(h_records, c->d_rec, static_cast<size_t>(c->shots) * c->rec_bytes,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_born)
    e = cudaMemcpy(h_born, c->d_born, sizeof(double) * c->shots * c->prog.n_meas,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_stats) {
    std::vector<int> mx(c->shots), nr(c->shots);
    std::vector<double> ds(c->shots), lp(c->shots);
    e = cudaMemcpy(mx.data(), c->d_maxchi, sizeof(int) * c->shots, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(nr.data(), c->d_near, sizeof(int) * c->shots, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ds.data(), c->d_disc, sizeof(double) * c->shots, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lp.data(), c->d_logp, sizeof(double) * c->shots, cudaMemcpyDeviceToHost);
    for (int64_t s = 0; s < c->shots && e == cudaSuccess; ++s)
      h_stats[s] = stn_shot_stats{mx[s], nr[s], ds[s], lp[s]};
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_read_records");
  return STN_OK;
}

const uint8_t *stn_device_records(const stn_ctx *c) { return c ? c->d_rec : nullptr; }

int32_t stn_num_detectors(const stn_ctx *c) { return c ? c->prog.n_det : -1; }

stn_status stn_read_detectors(stn_ctx *c, uint8_t *h_det, uint8_t *h_logical) {
  if (!c) return STN_EINVAL;
  if (c->shots < 1) return fail(c, STN_EINVAL, "no batch");
  cudaError_t e = stn::launch_detectors(c->d_rec, c->rec_bytes, c->shots, c->d_det_table, c->prog.n_det,
                                        c->d_logical, static_cast<int>(c->prog.logical.size()), c->d_det,
                                        c->d_obs, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "detector kernel");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  if (h_det)
    e = cudaMemcpy(h_det, c->d_det, static_cast<size_t>(c->shots) * ((c->prog.n_det + 7) / 8),
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_logical)
    e = cudaMemcpy(h_logical, c->d_obs, static_cast<size_t>(c->shots), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_read_detectors");
  return STN_OK;
}

stn_status stn_algorithmic_flops(stn_ctx *c, double *h_total) {
  if (!c || !h_total) return STN_EINVAL;
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  std::vector<double> f(c->max_shots);
  cudaError_t e = cudaMemcpy(f.data(), c->d_flops, sizeof(double) * c->max_shots, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_algorithmic_flops");
  double t = 0;
  for (double v : f) t += v;
  *h_total = t;
  return STN_OK;
}

stn_status stn_profile_counters(stn_ctx *c, double *h_out) {
  if (!c || !h_out) return STN_EINVAL;
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  std::vector<double> f(static_cast<size_t>(c->max_shots) * stn::kProfSlots);
  cudaError_t e = cudaMemcpy(f.data(), c->d_prof, sizeof(double) * f.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_profile_counters");
  for (int i = 0; i < stn::kProfSlots; ++i) h_out[i] = 0;
  for (size_t k = 0; k < f.size(); ++k) h_out[k % stn::kProfSlots] += f[k];
  return STN_OK;
}

stn_status stn_read_tableau(stn_ctx *c, int64_t shot, uint64_t *h_x, uint64_t *h_z,
                            uint8_t *h_phase) {
  if (!c || shot < 0 || shot >= c->shots) return fail(c, STN_EINVAL, "shot out of range");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  const size_t rows = 2 * c->n, words = rows * c->W;
  cudaError_t e = cudaSuccess;
  if (h_x) e = cudaMemcpy(h_x, c->d_tx + shot * words, sizeof(uint64_t) * words, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_z)
    e = cudaMemcpy(h_z, c->d_tz + shot * words, sizeof(uint64_t) * words, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_phase)
    e = cudaMemcpy(h_phase, c->d_tm + shot * rows, rows, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_read_tableau");
  return STN_OK;
}

stn_status stn_read_bonds(stn_ctx *c, int64_t shot, int32_t *h_bonds) {
  if (!c || shot < 0 || shot >= c->shots || !h_bonds) return fail(c, STN_EINVAL, "bad argument");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  std::vector<int> chi(c->n + 1);
  cudaError_t e = cudaMemcpy(chi.data(), c->d_chi + shot * (c->n + 1), sizeof(int) * (c->n + 1),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_read_bonds");
  for (int k = 0; k + 1 < c->n; ++k) h_bonds[k] = chi[k + 1];
  return STN_OK;
}

stn_status stn_read_site(stn_ctx *c, int64_t shot, int32_t k, void *h_site) {
  if (!c || shot < 0 || shot >= c->shots || k < 0 || k >= c->n || !h_site)
    return fail(c, STN_EINVAL, "bad argument");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  int dims[2];
  cudaError_t e = cudaMemcpy(dims, c->d_chi + shot * (c->n + 1) + k, sizeof(int) * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    const size_t bytes = c->elem * 2ull * dims[0] * dims[1];
    const char *src = static_cast<const char *>(c->d_mps) + c->elem * (shot * c->slab_elems + c->site_off[k]);
    e = cudaMemcpy(h_site, src, bytes, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_read_site");
  return STN_OK;
}

static cudaError_t launch_diag(stn_ctx *c, int what, int target, int cut, int nl, int letter, int grid) {
  stn::EngineParams p = params(c, 0, 0, c->d_theta);
  return c->cfg.precision == STN_PRECISION_C128
             ? stn::launch_diag_f64(p, what, target, cut, c->d_diag_q, nl, letter, c->d_diag, c->d_diag_count,
                                    grid, c->stream)
             : stn::launch_diag_f32(p, what, target, cut, c->d_diag_q, nl, letter, c->d_diag, c->d_diag_count,
                                    grid, c->stream);
}

stn_status stn_logical_expectation(stn_ctx *c, double *h_out) {
  if (!c || !h_out) return fail(c, STN_EINVAL, "bad argument");
  if (c->shots < 1) return fail(c, STN_EINVAL, "no batch");
  std::vector<int32_t> lq;
  const bool xmem = c->prog.basis == STN_BASIS_X;
  for (int q : c->prog.data)
    if ((!xmem && c->prog.xy[2 * q + 1] == 1) || (xmem && c->prog.xy[2 * q] == 1)) lq.push_back(q);
  cudaError_t e = cudaMemcpyAsync(c->d_diag_q, lq.data(), sizeof(int32_t) * lq.size(), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = launch_diag(c, 0, 0, 0, static_cast<int>(lq.size()), xmem ? 1 : 3,
                    static_cast<int>(std::min<int64_t>(c->grid, c->shots)));
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernel");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  e = cudaMemcpy(h_out, c->d_diag, sizeof(double) * c->shots, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_logical_expectation");
  return STN_OK;
}

stn_status stn_schmidt_values(stn_ctx *c, int64_t shot, int32_t cut, double *h_sig2, int32_t *h_count) {
  if (!c || !h_sig2 || !h_count || shot < 0 || shot >= c->shots || cut < 0 || cut > c->n - 2)
    return fail(c, STN_EINVAL, "bad argument");
  cudaError_t e = launch_diag(c, 1, static_cast<int>(shot), cut, 0, 0, 1);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernel");
  stn_status st = stn_sync(c);
  if (st != STN_OK) return st;
  int cnt = 0;
  e = cudaMemcpy(&cnt, c->d_diag_count, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && cnt > 0)
    e = cudaMemcpy(h_sig2, c->d_diag, sizeof(double) * cnt, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_schmidt_values");
  *h_count = cnt;
  return STN_OK;
}

stn_status stn_capture_batch(stn_ctx *c, int64_t shots, const double *d_theta) {
  if (!c) return STN_EINVAL;
  if (!c->stream) return fail(c, STN_EINVAL, "graph capture needs the context's own (non-default) stream");
  if (shots < 1 || shots > c->max_shots) return fail(c, STN_EINVAL, "shots must be 1..max_shots");
  if (!d_theta && c->K > 0) return fail(c, STN_EINVAL, "theta is NULL");
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->shots = shots;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
  stn::EngineParams p = params(c, 0, 0, d_theta ? d_theta : c->d_theta);
  p.shot_offset_dev = c->d_offset;
  cudaError_t le = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (le == cudaSuccess) le = stn::launch_init(c->cfg.precision, p, c->stream);
  const int grid = static_cast<int>(std::min<int64_t>(c->grid, shots));
  if (shots > grid) p.ticket = c->d_ticket;
  for (size_t st = 0; le == cudaSuccess && st + 1 < c->prog.step_begin.size(); ++st) {
    p.op_begin = c->prog.step_begin[st];
    p.op_end = c->prog.step_begin[st + 1];
    if (p.ticket) le = cudaMemsetAsync(c->d_ticket, 0, sizeof(int), c->stream);
    if (le == cudaSuccess) le = stn::launch_round(c->cfg.precision, p, grid, c->stream);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, le != cudaSuccess ? le : e, "capture");
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(c, e, "graph instantiate");
  }
  c->graph_shots = shots;
  return STN_OK;
}

stn_status stn_launch_captured(stn_ctx *c, uint64_t shot_offset) {
  if (!c) return STN_EINVAL;
  if (!c->graph) return fail(c, STN_EINVAL, "no captured batch: call stn_capture_batch first");
  c->shots = c->graph_shots;
  c->shot_offset = shot_offset;
  cudaError_t e = cudaMemcpyAsync(c->d_offset, &c->shot_offset, sizeof(uint64_t), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(c->graph, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  return STN_OK;
}

stn_status stn_sample_shots(stn_ctx *c, int64_t shots, uint64_t shot_offset, const double *h_theta,
                            uint8_t *h_records, double *h_born, stn_shot_stats *h_stats) {
  stn_status st = stn_begin_batch(c, shots, shot_offset);
  for (int r = 0; st == STN_OK && r <= c->cfg.rounds; ++r) st = stn_apply_round(c, r, h_theta);
  if (st != STN_OK) return st;
  return stn_read_records(c, h_records, h_born, h_stats);
}


stn_status stn_logprob_grad(stn_ctx *c, uint64_t shot_offset, int64_t n_rec, const uint8_t *h_records,
                            const double *h_theta, double *h_logp, double *h_grad) {
  if (!c) return STN_EINVAL;
  if (n_rec < 1 || n_rec > c->max_shots || !h_records || !h_logp || !h_grad || (!h_theta && c->K > 0))
    return fail(c, STN_EINVAL, "stn_logprob_grad: bad argument");
  for (int k = 0; k < c->K; ++k)
    if (!std::isfinite(h_theta[k])) return fail(c, STN_EINVAL, "theta must be finite");
  const int n_ops = static_cast<int>(c->prog.ops.size());
  std::vector<int32_t> rot_ord(n_ops, -1);
  int n_rot = 0;
  for (int i = 0; i < n_ops; ++i)
    if (c->prog.ops[i].kind == stn::OP_ROT) rot_ord[i] = n_rot++;
  const size_t phi_bytes = c->elem * static_cast<size_t>(n_rec) * std::max(1, n_rot) * c->slab_elems;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "memory info");
  if (phi_bytes > free_b / 10 * 8)
    return fail(c, STN_ENOMEM, "stn_logprob_grad: the states after every rotation do not fit device memory");
  AdjointBuffers buf;
  uint8_t *d_forced = nullptr;
  uint64_t *d_px = nullptr, *d_pz = nullptr;
  int32_t *d_info = nullptr, *d_rot = nullptr;
  void *d_phi = nullptr;
  int *d_phi_chi = nullptr;
  double *d_grad = nullptr;
  const size_t tape = static_cast<size_t>(n_rec) * n_ops;
  bool ok = buf.get(&d_forced, static_cast<size_t>(n_rec) * c->rec_bytes) &&
            buf.get(&d_px, sizeof(uint64_t) * tape * c->W) && buf.get(&d_pz, sizeof(uint64_t) * tape * c->W) &&
            buf.get(&d_info, sizeof(int32_t) * tape * stn::kTapeInts) &&
            buf.get(&d_rot, sizeof(int32_t) * n_ops) && buf.get(&d_phi, phi_bytes) &&
            buf.get(&d_phi_chi, sizeof(int) * static_cast<size_t>(n_rec) * std::max(1, n_rot) * (c->n + 1)) &&
            buf.get(&d_grad, sizeof(double) * std::max(1, c->K));
  if (!ok) return fail(c, STN_ENOMEM, "stn_logprob_grad: device allocation failed");
  stn_status st = stn_begin_batch(c, n_rec, shot_offset);
  if (st != STN_OK) return st;
  cudaError_t e = cudaMemcpyAsync(d_forced, h_records, static_cast<size_t>(n_rec) * c->rec_bytes,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rot, rot_ord.data(), sizeof(int32_t) * n_ops, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && c->K > 0)
    e = cudaMemcpyAsync(c->d_theta, h_theta, sizeof(double) * c->K, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_grad, 0, sizeof(double) * std::max(1, c->K), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_logprob_grad copies");
  stn::EngineParams p = params(c, 0, n_ops, c->d_theta);
  p.forced = d_forced;
  p.tape_px = d_px;
  p.tape_pz = d_pz;
  p.tape_info = d_info;
  p.phi_store = d_phi;
  p.phi_chi = d_phi_chi;
  p.rot_ord = d_rot;
  p.n_ops_total = n_ops;
  p.n_rot = n_rot;
  const int grid = static_cast<int>(std::min<int64_t>(c->grid, n_rec));
  e = stn::launch_round(c->cfg.precision, p, grid, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint forward");
  st = stn_sync(c);
  if (st != STN_OK) return st;
  e = cudaMemcpy(h_logp, c->d_logp, sizeof(double) * n_rec, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_logprob_grad logp");
  e = c->cfg.precision == STN_PRECISION_C128 ? stn::launch_adjoint_f64(p, d_grad, grid, c->stream)
                                             : stn::launch_adjoint_f32(p, d_grad, grid, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint backward");
  st = stn_sync(c);
  if (st != STN_OK) return st;
  e = cudaMemcpy(h_grad, d_grad, sizeof(double) * c->K, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stn_logprob_grad grad");
  return STN_OK;
}

stn_status stn_dense_qr_q(int32_t precision, int32_t m, int32_t n, void *d_b, void *d_q, void *d_work,
                          void *cuda_stream) {
  if ((precision != 0 && precision != 1) || m < 1 || n < 1 || m > 1024 || !d_b || !d_q || !d_work)
    return STN_EINVAL;
  cudaError_t e = stn::launch_dense_check(precision, 2, m, n, d_b, d_q, d_work, 0,
                                          static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

stn_status stn_dense_qr(int32_t precision, int32_t m, int32_t n, void *d_b, void *cuda_stream) {
  if ((precision != 0 && precision != 1) || m < 1 || n < 1 || m > 1024 || !d_b) return STN_EINVAL;
  cudaError_t e = stn::launch_dense_check(precision, 0, m, n, d_b, nullptr, nullptr, 0,
                                          static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

stn_status stn_dense_svd(int32_t precision, int32_t m, int32_t n, void *d_c, void *d_v, void *d_sig2,
                         int32_t in_shared, void *cuda_stream) {
  if ((precision != 0 && precision != 1) || m < 1 || n < 1 || n > 512 || !d_c || !d_v || !d_sig2)
    return STN_EINVAL;
  if (in_shared == 1 && m * n + n * n > stn::svd_smem_elems(precision)) return STN_EINVAL;
  if (in_shared < 0 || in_shared > 3 || (in_shared >= 2 && 2 * m + 4 > stn::svd_smem_elems(precision)))
    return STN_EINVAL;
  if (in_shared == 3 && (m > 1024 || 2 * n + 4 > stn::svd_smem_elems(precision))) return STN_EINVAL;
  cudaError_t e = stn::launch_dense_check(precision, 1, m, n, d_c, d_v, d_sig2, in_shared,
                                          static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

stn_status stn_dense_cgemm(int32_t precision, int32_t gemm_units, int32_t op_a, int32_t op_b, int32_t m,
                           int32_t n, int32_t k, const double *alpha, const void *d_a, int32_t lda,
                           const void *d_b, int32_t ldb, const double *beta, void *d_c, int32_t ldc,
                           int32_t *d_status, void *cuda_stream) {
  if ((precision != 0 && precision != 1) || (gemm_units != STN_GEMM_TENSOR && gemm_units != STN_GEMM_FMA) ||
      (op_a != 0 && op_a != 1) || (op_b != 0 && op_b != 1))
    return STN_EINVAL;
  if (m < 1 || n < 1 || k < 1 || m > 4096 || n > 4096 || k > 4096) return STN_EINVAL;
  if (lda < (op_a ? m : k) || ldb < (op_b ? k : n) || ldc < n) return STN_EINVAL;
  if (!alpha || !beta || !d_a || !d_b || !d_c || !d_status) return STN_EINVAL;
  const int use_tc = precision == 1 && gemm_units == STN_GEMM_TENSOR ? 1 : 0;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = precision == 0
                      ? stn::launch_dense_gemm_f64(op_a, op_b, m, n, k, alpha, d_a, lda, d_b, ldb, beta, d_c, ldc,
                                                   use_tc, d_status, s)
                      : stn::launch_dense_gemm_f32(op_a, op_b, m, n, k, alpha, d_a, lda, d_b, ldb, beta, d_c, ldc,
                                                   use_tc, d_status, s);
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

stn_status stn_dense_svd_noalloc(int32_t precision, int32_t m, int32_t n, const void *d_c, void *d_v,
                                 void *d_sig2, void *cuda_stream) {
  if ((precision != 0 && precision != 1) || m < 1 || n < 1 || m > 1024 || n > 512 || !d_c || !d_v || !d_sig2)
    return STN_EINVAL;
  if (2 * m + 4 > stn::svd_smem_elems(precision) || 2 * n + 4 > stn::svd_smem_elems(precision))
    return STN_EINVAL;
  const size_t elem = precision == 0 ? 16 : 8;
  if (static_cast<size_t>(m) * n * elem > stn::noalloc_scratch_bytes()) return STN_EOVERFLOW;
  cudaError_t e = stn::launch_svd_noalloc(precision, m, n, d_c, d_v, d_sig2,
                                          static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

stn_status stn_philox_uniforms(uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                               uint32_t event_offset, int32_t n_events, double *d_out,
                               void *cuda_stream) {
  if (n_shots < 0 || n_events < 0 || (!d_out && n_shots * n_events > 0)) return STN_EINVAL;
  cudaError_t e = stn::launch_philox(seed, shot_offset, n_shots, event_offset, n_events, d_out,
                                     static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? STN_OK : STN_ECUDA;
}

}  // extern "C"
