// Host side of the libdcs C ABI (declared in include/dcs.h): context and arena layout,
// chunk construction, the per-chunk tables (with the FP64 operator-Schmidt split of every
// two-qubit gate) and the single-/multi-path drivers of Alg. 1 and Alg. 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dcs_kernels.cuh"
#include "dcs_plan.h"
#include "dcs_tables.h"


using namespace dcs;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kProgBytes = 32ull << 20;  // device copy of one call's tables

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t mps0, mps1, env, offs, bonds, centre, ketbuf, p, F, rr, creg, flags, shot, order, count,
      status, plan, counters, prog, work, total;
  bool big;
  size_t work_stride;
  int chi_cap;
  int dmax;  // MPO bond cap of a chunk (4 per sub-layer, multiplied over sub-layers)
  size_t mps_slot_stride, env_slot_stride;
};

bool valid_cfg(const dcs_config* c) {
  return c && c->n_qubits >= 1 && c->n_qubits <= DCS_MAX_QUBITS && c->chi_max >= 1 &&
         c->sweeps >= 1 && c->n_slots >= 1 && c->n_cbits >= 0 && c->n_cbits <= 64 * DCS_CWORDS &&
         c->tol >= 0.0 && c->chunk_k >= 0 && c->chunk_layers >= 0 &&
         c->chunk_layers <= DCS_MAX_CHUNK_LAYERS &&
         (c->precision == DCS_PREC_FP32 || c->precision == DCS_PREC_TF32X3 ||
          c->precision == DCS_PREC_BF16X3) &&
         c->kernel_path >= DCS_PATH_AUTO && c->kernel_path <= DCS_PATH_GLOBAL;
}

// shared-memory tiles or the global work area; false if chi_max cannot be held
// (chunks of several layers: the global work area only)
bool pick_path(const dcs_config* c, bool& big) {
  if (c->chi_max > DCS_MAX_CHI) return false;
  const bool multi = c->chunk_layers > 1;
  if (c->kernel_path == DCS_PATH_SHARED) {
    big = false;
    return !multi && fused_chi(c->chi_max) != 0;
  }
  big = multi || c->kernel_path == DCS_PATH_GLOBAL || fused_chi(c->chi_max) == 0;
  return true;
}

Layout make_layout(const dcs_config* c) {
  Layout L{};
  const size_t n = (size_t)c->n_qubits, S = (size_t)c->n_slots;
  pick_path(c, L.big);
  L.chi_cap = L.big ? big_chi(c->chi_max) : fused_chi(c->chi_max);
  L.dmax = chunk_dmax(c->chunk_layers);
  L.work_stride = L.big ? big_work_elems(L.chi_cap, L.dmax) : 0;
  layout_offsets((int)n, L.chi_cap, L.dmax, nullptr, nullptr, &L.mps_slot_stride,
                 &L.env_slot_stride);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.mps0 = take(S * L.mps_slot_stride * sizeof(float2));
  L.mps1 = take(S * L.mps_slot_stride * sizeof(float2));
  L.env = take(S * L.env_slot_stride * sizeof(float2));
  L.offs = take(2 * (n + 1) * sizeof(size_t));
  L.bonds = take(S * 2 * (n + 1) * sizeof(int32_t));
  L.centre = take(S * sizeof(int32_t));
  L.ketbuf = take(S * sizeof(int32_t));
  L.p = take(S * sizeof(double));
  L.F = take(S * sizeof(double));
  L.rr = take(S * 2 * sizeof(double));
  L.creg = take(S * DCS_CWORDS * sizeof(uint64_t));
  L.flags = take(S * sizeof(uint32_t));
  L.shot = take(S * sizeof(uint64_t));
  L.order = take(S * sizeof(int32_t));
  L.count = take(sizeof(int32_t));
  L.status = take(sizeof(int32_t));
  L.plan = take((PLAN_HDR + 4 * S) * sizeof(int32_t));
  L.counters = take(2 * sizeof(unsigned long long));
  L.prog = take(kProgBytes);
  L.work = take(S * L.work_stride * sizeof(float2));
  L.total = off;
  return L;
}

// ----------------------------------------------------------------------------- program
struct Program {
  std::vector<DLayer> layers;
  std::vector<DBlock> blocks;
  std::vector<DGate1> g1;
  std::vector<DCond> conds;
  std::vector<DMeas> meas;
  std::vector<Step> steps;
  bool overflow() const { return false; }
};

// a chunk's sub-layers (add_chunk) and the step that launches it; no more sub-layers than
// the context's chunk_layers
std::string add_layer(Program& P, int n, const std::vector<dcs_op>& gates, int max_sub) {
  if ((int)split_sublayers(gates.data(), (int)gates.size(), n).size() > max_sub)
    return "a qubit carries more two-qubit gates than the chunk has layers";
  const char* e = add_chunk(P, n, gates.data(), (int)gates.size());
  return e ? e : "";
}

}  // namespace

// ----------------------------------------------------------------------------- context
struct dcs_ctx_s {
  dcs_config cfg{};
  Layout lay{};
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  DevCtx dev{};
  char* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
  std::string err;
  uint64_t launches = 0;
  uint64_t uploaded = 0;
  int multipath = 0;
  double prune_pmin = 0.0;  // adaptive pruning threshold of branch splits (0: off)
  // Upper bound on every bond dimension any slot can have, per bond, tracked from the
  // circuit alone: a two-qubit block on (q, q+1) makes bond q+1 at most
  // min(chi_max, 2 ub[q], 2 ub[q+2], 2^min(q+1, n-q-1)) (the truncated SVD of a
  // (2 chi_q) x (2 chi_{q+2}) matrix); QR steps, measurements and single-qubit gates never
  // raise a bond.  The shared-memory tile of a launch is the smallest one above this bound.
  std::vector<int> ub;
  std::vector<size_t> site_off, env_off;  // host copy of the bond-sized layout offsets
  int tile() const {
    int m = 1;
    for (int v : ub) m = std::max(m, v);
    return fused_chi(m);
  }
};

namespace {

dcs_status_t fail(dcs_ctx_t c, dcs_status_t s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

dcs_status_t cuda_check(dcs_ctx_t c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DCS_OK;
  return fail(c, DCS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Copy a program's tables to the device program region; fills the device pointers.
struct DevProg {
  const DLayer* layers;
  const DBlock* blocks;
  const DGate1* g1;
  const DCond* conds;
  const DMeas* meas;
  const uint8_t* bytes;
};

// The pinned host staging buffer, at least `total` bytes, with no copy still reading it.
dcs_status_t ensure_stage(dcs_ctx_t c, size_t total) {
  if (c->stage_pending) {
    cudaError_t e = cudaEventSynchronize(c->stage_done);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaEventSynchronize");
    c->stage_pending = false;
  }
  if (total > c->stage_bytes) {
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMallocHost(&c->stage, total);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaMallocHost");
    c->stage_bytes = total;
  }
  return DCS_OK;
}

dcs_status_t upload(dcs_ctx_t c, const Program& P, const std::vector<uint8_t>& extra, DevProg& out) {
  size_t off = 0;
  auto sz = [&](size_t b) {
    const size_t o = off;
    off = align_up(off + b);
    return o;
  };
  const size_t oL = sz(P.layers.size() * sizeof(DLayer));
  const size_t oB = sz(P.blocks.size() * sizeof(DBlock));
  const size_t oG = sz(P.g1.size() * sizeof(DGate1));
  const size_t oC = sz(P.conds.size() * sizeof(DCond));
  const size_t oM = sz(P.meas.size() * sizeof(DMeas));
  const size_t oX = sz(extra.size());
  const size_t total = off;
  if (total > kProgBytes) return fail(c, DCS_ERR_OOM, "circuit tables exceed the program region");
  if (dcs_status_t st = ensure_stage(c, total); st != DCS_OK) return st;
  auto put = [&](size_t o, const void* src, size_t b) {
    if (b) std::memcpy(c->stage + o, src, b);
  };
  put(oL, P.layers.data(), P.layers.size() * sizeof(DLayer));
  put(oB, P.blocks.data(), P.blocks.size() * sizeof(DBlock));
  put(oG, P.g1.data(), P.g1.size() * sizeof(DGate1));
  put(oC, P.conds.data(), P.conds.size() * sizeof(DCond));
  put(oM, P.meas.data(), P.meas.size() * sizeof(DMeas));
  put(oX, extra.data(), extra.size());
  char* dprog = c->arena + c->lay.prog;
  if (total) {
    cudaError_t e = cudaMemcpyAsync(dprog, c->stage, total, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaMemcpyAsync(tables)");
    cudaEventRecord(c->stage_done, c->stream);
    c->stage_pending = true;
    c->uploaded += total;
  }
  out.layers = reinterpret_cast<const DLayer*>(dprog + oL);
  out.blocks = reinterpret_cast<const DBlock*>(dprog + oB);
  out.g1 = reinterpret_cast<const DGate1*>(dprog + oG);
  out.conds = reinterpret_cast<const DCond*>(dprog + oC);
  out.meas = reinterpret_cast<const DMeas*>(dprog + oM);
  out.bytes = reinterpret_cast<const uint8_t*>(dprog + oX);
  return DCS_OK;
}

dcs_status_t post_launch(dcs_ctx_t c, const char* what) {
  cudaError_t e = cudaGetLastError();
  return cuda_check(c, e, what);
}

dcs_status_t check_gate(dcs_ctx_t c, const dcs_op& o) {
  const int n = c->cfg.n_qubits;
  if (o.kind == DCS_OP_GATE1) {
    if (o.q0 < 0 || o.q0 >= n) return fail(c, DCS_ERR_INVALID, "qubit out of range");
  } else if (o.kind == DCS_OP_GATE2) {
    if (o.q0 < 0 || o.q0 >= n || o.q1 < 0 || o.q1 >= n || std::abs(o.q0 - o.q1) != 1)
      return fail(c, DCS_ERR_INVALID, "two-qubit gates must act on neighbouring qubits");
  } else if (o.kind == DCS_OP_MEASURE || o.kind == DCS_OP_RESET) {
    if (o.q0 < 0 || o.q0 >= n) return fail(c, DCS_ERR_INVALID, "qubit out of range");
    if (o.cbit < 0 || o.cbit >= c->cfg.n_cbits) return fail(c, DCS_ERR_INVALID, "cbit out of range");
  } else {
    return fail(c, DCS_ERR_INVALID, "unknown operation kind");
  }
  if (!cond_valid(o.cond))
    return fail(c, DCS_ERR_INVALID, "unknown condition op");
  if ((o.kind == DCS_OP_MEASURE || o.kind == DCS_OP_RESET) && o.cond.op != DCS_COND_NONE)
    return fail(c, DCS_ERR_INVALID, "measurements cannot be classically controlled");
  return DCS_OK;
}

void grow_bounds(dcs_ctx_t c, const Program& P, const DLayer& L) {
  const int n = c->cfg.n_qubits;
  std::vector<int>& ub = c->ub;
  for (int b = 0; b < L.n_blocks; ++b) {
    const int q = P.blocks[L.blk_off + b].q;
    const int e = std::min(q + 1, n - q - 1);
    const int hil = e >= 30 ? (1 << 30) : (1 << e);
    ub[q + 1] = std::min({c->cfg.chi_max, 2 * ub[q], 2 * ub[q + 2], hil});
  }
}

dcs_status_t run_steps(dcs_ctx_t c, const Program& P, int max_branches,
                       double* fid_out) {
  DevProg dp;
  std::vector<uint8_t> none;
  dcs_status_t st = upload(c, P, none, dp);
  if (st != DCS_OK) return st;
  for (const Step& s : P.steps) {
    if (s.kind == 0) {
      for (int l = 0; l < s.n; ++l) grow_bounds(c, P, P.layers[s.idx + l]);
      launch_compress(c->dev, c->tile(), dp.layers + s.idx, s.n, dp.blocks, dp.g1, dp.conds,
                      fid_out, c->stream);
      c->launches++;
      if ((st = post_launch(c, "compress")) != DCS_OK) return st;
    } else if (!c->multipath) {
      launch_measure(c->dev, c->tile(), dp.meas + s.idx, s.n, MEAS_SAMPLE, nullptr, nullptr,
                     c->stream);
      c->launches++;
      if ((st = post_launch(c, "measure")) != DCS_OK) return st;
    } else {
      for (int i = 0; i < s.n; ++i) {
        const DMeas& m = P.meas[s.idx + i];
        launch_measure(c->dev, c->tile(), dp.meas + s.idx + i, 1, MEAS_PROB, nullptr, nullptr,
                       c->stream);
        c->launches++;
        int l = 0;
        launch_branch_split(c->dev, m.q, m.cbit, 1e-12, max_branches, c->prune_pmin, c->stream,
                            &l);
        c->launches += l;
        if ((st = post_launch(c, "branch split")) != DCS_OK) return st;
      }
    }
  }
  return DCS_OK;
}

}  // namespace

extern "C" {

size_t dcs_arena_bytes(const dcs_config* cfg) {
  bool big;
  if (!valid_cfg(cfg) || !pick_path(cfg, big)) return 0;
  return make_layout(cfg).total;
}

dcs_status_t dcs_create(dcs_ctx_t* out, const dcs_config* cfg, void* dev_arena, size_t bytes,
                        dcs_stream_t stream) {
  if (!out) return DCS_ERR_INVALID;
  *out = nullptr;
  if (!valid_cfg(cfg)) return DCS_ERR_INVALID;
  bool big;
  if (!pick_path(cfg, big)) return DCS_ERR_UNSUPPORTED;
  const Layout lay = make_layout(cfg);
  if (!dev_arena || bytes < lay.total) return DCS_ERR_OOM;
  if (reinterpret_cast<uintptr_t>(dev_arena) % kAlign) return DCS_ERR_INVALID;
  dcs_ctx_s* c = new dcs_ctx_s();
  c->cfg = *cfg;
  c->lay = lay;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->arena = static_cast<char*>(dev_arena);
  DevCtx& d = c->dev;
  d.n = cfg->n_qubits;
  d.chi_cap = lay.chi_cap;
  d.dmax = lay.dmax;
  d.n_slots = cfg->n_slots;
  d.mps_slot_stride = lay.mps_slot_stride;
  d.env_slot_stride = lay.env_slot_stride;
  char* a = c->arena;
  d.mps[0] = reinterpret_cast<float2*>(a + lay.mps0);
  d.mps[1] = reinterpret_cast<float2*>(a + lay.mps1);
  d.env = reinterpret_cast<float2*>(a + lay.env);
  d.site_off = reinterpret_cast<const size_t*>(a + lay.offs);
  d.env_off = d.site_off + (cfg->n_qubits + 1);
  d.bonds = reinterpret_cast<int32_t*>(a + lay.bonds);
  d.centre = reinterpret_cast<int32_t*>(a + lay.centre);
  d.ketbuf = reinterpret_cast<int32_t*>(a + lay.ketbuf);
  d.p = reinterpret_cast<double*>(a + lay.p);
  d.F = reinterpret_cast<double*>(a + lay.F);
  d.rr = reinterpret_cast<double*>(a + lay.rr);
  d.creg = reinterpret_cast<uint64_t*>(a + lay.creg);
  d.flags = reinterpret_cast<uint32_t*>(a + lay.flags);
  d.shot = reinterpret_cast<uint64_t*>(a + lay.shot);
  d.order = reinterpret_cast<int32_t*>(a + lay.order);
  d.count = reinterpret_cast<int32_t*>(a + lay.count);
  d.status = reinterpret_cast<int32_t*>(a + lay.status);
  d.plan = reinterpret_cast<int32_t*>(a + lay.plan);
  d.counters = reinterpret_cast<unsigned long long*>(a + lay.counters);
  d.work = lay.big ? reinterpret_cast<float2*>(a + lay.work) : nullptr;
  d.use_tc = !lay.big ? 0
             : cfg->precision == DCS_PREC_TF32X3 ? 1
             : cfg->precision == DCS_PREC_BF16X3 ? 2 : 0;
  d.work_stride = lay.work_stride;
  d.seed = cfg->seed;
  d.chi_max = cfg->chi_max;
  d.tol = cfg->tol;
  d.sweeps = cfg->sweeps;
  c->ub.assign(cfg->n_qubits + 1, 1);
  c->site_off.assign(cfg->n_qubits + 1, 0);
  c->env_off.assign(cfg->n_qubits + 1, 0);
  size_t me = 0, ee = 0;
  layout_offsets(cfg->n_qubits, lay.chi_cap, lay.dmax, c->site_off.data(), c->env_off.data(), &me,
                 &ee);
  if (cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return DCS_ERR_CUDA;
  }
  *out = c;
  return DCS_OK;
}

dcs_status_t dcs_destroy(dcs_ctx_t c) {
  if (!c) return DCS_ERR_INVALID;
  if (c->stage_pending) cudaEventSynchronize(c->stage_done);
  if (c->stage) cudaFreeHost(c->stage);
  if (c->stage_done) cudaEventDestroy(c->stage_done);
  delete c;
  return DCS_OK;
}

const char* dcs_last_error(dcs_ctx_t c) { return c ? c->err.c_str() : "null context"; }

uint64_t dcs_kernel_launches(dcs_ctx_t c) { return c ? c->launches : 0; }

uint64_t dcs_bytes_uploaded(dcs_ctx_t c) { return c ? c->uploaded : 0; }

dcs_status_t dcs_get_counters(dcs_ctx_t c, uint64_t* compressions, uint64_t* sweeps) {
  if (!c) return DCS_ERR_INVALID;
  dcs_status_t st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronize");
  if (st != DCS_OK) return st;
  unsigned long long v[2] = {0, 0};
  cudaMemcpy(v, c->dev.counters, sizeof(v), cudaMemcpyDeviceToHost);
  if (compressions) *compressions = v[0];
  if (sweeps) *sweeps = v[1];
  return cuda_check(c, cudaGetLastError(), "counters");
}

dcs_status_t dcs_init_state(dcs_ctx_t c, int n_active, int multipath, uint64_t shot0) {
  if (!c) return DCS_ERR_INVALID;
  if (n_active < 1 || n_active > c->cfg.n_slots) return fail(c, DCS_ERR_INVALID, "n_active out of range");
  if (multipath && n_active != 1) return fail(c, DCS_ERR_INVALID, "multi-path starts from one branch");
  c->multipath = multipath ? 1 : 0;
  c->ub.assign(c->cfg.n_qubits + 1, 1);
  launch_init(c->dev, n_active, c->multipath, shot0, c->stream);
  c->launches += 2;
  return post_launch(c, "init");
}

dcs_status_t dcs_fork_shots(dcs_ctx_t c, int n_active) {
  if (!c) return DCS_ERR_INVALID;
  if (c->multipath) return fail(c, DCS_ERR_INVALID, "forking shots needs single-path mode");
  if (n_active < 1 || n_active > c->cfg.n_slots) return fail(c, DCS_ERR_INVALID, "n_active out of range");
  launch_fork_shots(c->dev, n_active, c->stream);
  c->launches += 2;
  return post_launch(c, "fork shots");
}

dcs_status_t dcs_apply_layer(dcs_ctx_t c, const dcs_op* gates, int n_gates, double* fid_out) {
  if (!c || (n_gates > 0 && !gates)) return fail(c, DCS_ERR_INVALID, "null argument");
  std::vector<dcs_op> g(gates, gates + n_gates);
  for (const dcs_op& o : g) {
    if (o.kind != DCS_OP_GATE1 && o.kind != DCS_OP_GATE2)
      return fail(c, DCS_ERR_INVALID, "dcs_apply_layer takes gates only");
    dcs_status_t st = check_gate(c, o);
    if (st != DCS_OK) return st;
  }
  if (g.empty()) return DCS_OK;
  Program P;
  std::string e = add_layer(P, c->cfg.n_qubits, g, std::max(1, c->cfg.chunk_layers));
  if (!e.empty()) return fail(c, DCS_ERR_INVALID, e);
  return run_steps(c, P, 0, fid_out);
}

static dcs_status_t measure_common(dcs_ctx_t c, int qubit, int cbit, uint64_t ord, int mode,
                                   const uint8_t* forced, double* p0_out) {
  if (!c) return DCS_ERR_INVALID;
  if (qubit < 0 || qubit >= c->cfg.n_qubits) return fail(c, DCS_ERR_INVALID, "qubit out of range");
  if (mode != MEAS_PROB && (cbit < 0 || cbit >= c->cfg.n_cbits))
    return fail(c, DCS_ERR_INVALID, "cbit out of range");
  Program P;
  P.meas.push_back({qubit, cbit, ord});
  std::vector<uint8_t> extra;
  if (forced) extra.assign(forced, forced + c->cfg.n_slots);
  DevProg dp;
  dcs_status_t st = upload(c, P, extra, dp);
  if (st != DCS_OK) return st;
  launch_measure(c->dev, c->tile(), dp.meas, 1, mode, forced ? dp.bytes : nullptr, p0_out,
                 c->stream);
  c->launches++;
  return post_launch(c, "measure");
}

dcs_status_t dcs_measure_prob(dcs_ctx_t c, int qubit, double* p0_out) {
  return measure_common(c, qubit, 0, 0, MEAS_PROB, nullptr, p0_out);
}

dcs_status_t dcs_measure_sample(dcs_ctx_t c, int qubit, int cbit, uint64_t meas_idx) {
  if (c && c->multipath) return fail(c, DCS_ERR_INVALID, "sampling is single-path only");
  return measure_common(c, qubit, cbit, meas_idx, MEAS_SAMPLE, nullptr, nullptr);
}

dcs_status_t dcs_collapse(dcs_ctx_t c, int qubit, int cbit, const uint8_t* outcome) {
  if (!c || !outcome) return fail(c, DCS_ERR_INVALID, "null argument");
  return measure_common(c, qubit, cbit, 0, MEAS_FORCED, outcome, nullptr);
}

dcs_status_t dcs_branch_split(dcs_ctx_t c, int qubit, int cbit, double eps) {
  if (!c) return DCS_ERR_INVALID;
  if (!c->multipath) return fail(c, DCS_ERR_INVALID, "branch split needs multi-path mode");
  dcs_status_t st = measure_common(c, qubit, cbit, 0, MEAS_PROB, nullptr, nullptr);
  if (st != DCS_OK) return st;
  int l = 0;
  launch_branch_split(c->dev, qubit, cbit, eps, 0, c->prune_pmin, c->stream, &l);
  c->launches += l;
  return post_launch(c, "branch split");
}

dcs_status_t dcs_set_pruning(dcs_ctx_t c, double p_min) {
  if (!c || !(p_min >= 0.0) || p_min >= 1.0) return fail(c, DCS_ERR_INVALID, "p_min must lie in [0, 1)");
  c->prune_pmin = p_min;
  return DCS_OK;
}

dcs_status_t dcs_branch_topk(dcs_ctx_t c, int M) {
  if (!c || M < 1) return fail(c, DCS_ERR_INVALID, "M must be >= 1");
  if (!c->multipath) return fail(c, DCS_ERR_INVALID, "TopK needs multi-path mode");
  launch_branch_topk(c->dev, M, c->stream);
  c->launches++;
  return post_launch(c, "topk");
}

dcs_status_t dcs_branch_keep(dcs_ctx_t c, const uint8_t* keep, int n) {
  if (!c || n < 0 || (n > 0 && !keep)) return fail(c, DCS_ERR_INVALID, "null mask or negative length");
  if (!c->multipath) return fail(c, DCS_ERR_INVALID, "branch keep needs multi-path mode");
  if (n > c->cfg.n_slots) return fail(c, DCS_ERR_INVALID, "mask longer than the branch pool");
  Program P;
  std::vector<uint8_t> mask(keep, keep + n);
  DevProg dp;
  dcs_status_t st = upload(c, P, mask, dp);
  if (st != DCS_OK) return st;
  launch_branch_keep(c->dev, dp.bytes, n, c->stream);
  c->launches++;
  return post_launch(c, "branch keep");
}

dcs_status_t dcs_topk_select_global(const double* p, int n, int M, double p_min, uint8_t* keep) {
  if (n < 0 || M < 1 || (n > 0 && (!p || !keep)) || !(p_min >= 0.0) || p_min >= 1.0)
    return DCS_ERR_INVALID;
  double pmax = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(p[i] >= 0.0) || !std::isfinite(p[i])) return DCS_ERR_INVALID;
    pmax = std::max(pmax, p[i]);
  }
  if (n == 0) return DCS_OK;
  // the key of dcs_branch_topk, with the maximum over every rank's branches
  std::vector<long long> key(n);
  for (int i = 0; i < n; ++i)
    key[i] = pmax > 0.0 ? (long long)std::floor(p[i] / (1e-5 * pmax) + 0.5) : 0;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return key[a] > key[b]; });
  for (int i = 0; i < n; ++i) keep[i] = n <= M ? 1 : 0;
  if (n > M)
    for (int r = 0; r < M; ++r) keep[ord[r]] = 1;
  if (p_min > 0.0)
    for (int i = 0; i < n; ++i)
      if (keep[i] && p[i] < p_min && i != ord[0]) keep[i] = 0;
  return DCS_OK;
}

dcs_status_t dcs_get_results(dcs_ctx_t c, double* p, double* fid, uint64_t* cbits, int* n_active,
                             uint8_t* flags) {
  if (!c) return DCS_ERR_INVALID;
  dcs_status_t st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronize");
  if (st != DCS_OK) return st;
  // every per-slot array comes down into the pinned stage in one batch of async copies on
  // the context's stream, then is gathered into the caller's buffers in list order
  const size_t S = (size_t)c->cfg.n_slots;
  size_t off = 0;
  auto region = [&](size_t b) {
    const size_t o = off;
    off = align_up(off + b);
    return o;
  };
  const size_t oH = region(2 * sizeof(int));
  const size_t oO = region(S * sizeof(int));
  const size_t oP = region(p ? S * sizeof(double) : 0);
  const size_t oF = region(fid ? S * sizeof(double) : 0);
  const size_t oC = region(cbits ? S * DCS_CWORDS * sizeof(uint64_t) : 0);
  const size_t oL = region(flags ? S * sizeof(uint32_t) : 0);
  if ((st = ensure_stage(c, off)) != DCS_OK) return st;
  char* h = c->stage;
  cudaError_t e = cudaSuccess;
  auto get = [&](size_t o, const void* src, size_t b) {
    if (b && e == cudaSuccess) e = cudaMemcpyAsync(h + o, src, b, cudaMemcpyDeviceToHost, c->stream);
  };
  get(oH, c->dev.count, sizeof(int));
  get(oH + sizeof(int), c->dev.status, sizeof(int));
  get(oO, c->dev.order, S * sizeof(int));
  if (p) get(oP, c->dev.p, S * sizeof(double));
  if (fid) get(oF, c->dev.F, S * sizeof(double));
  if (cbits) get(oC, c->dev.creg, S * DCS_CWORDS * sizeof(uint64_t));
  if (flags) get(oL, c->dev.flags, S * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if ((st = cuda_check(c, e, "result copy")) != DCS_OK) return st;
  const int cnt = reinterpret_cast<const int*>(h + oH)[0];
  const int status = reinterpret_cast<const int*>(h + oH)[1];
  const int* order = reinterpret_cast<const int*>(h + oO);
  // the caller's buffers hold n_slots entries: a count or slot index outside the pool can
  // only come from corrupted device state, and is reported instead of written out
  if (cnt < 0 || (size_t)cnt > S) return fail(c, DCS_ERR_CUDA, "active count out of range");
  for (int i = 0; i < cnt; ++i)
    if (order[i] < 0 || (size_t)order[i] >= S)
      return fail(c, DCS_ERR_CUDA, "slot list out of range");
  if (n_active) *n_active = cnt;
  for (int i = 0; i < cnt; ++i) {
    const size_t slot = (size_t)order[i];
    if (p) p[i] = reinterpret_cast<const double*>(h + oP)[slot];
    if (fid) fid[i] = reinterpret_cast<const double*>(h + oF)[slot];
    if (cbits) {
      const uint64_t* src = reinterpret_cast<const uint64_t*>(h + oC) + slot * DCS_CWORDS;
      for (int w = 0; w < DCS_CWORDS; ++w) cbits[(size_t)i * DCS_CWORDS + w] = src[w];
    }
    if (flags) flags[i] = (uint8_t)reinterpret_cast<const uint32_t*>(h + oL)[slot];
  }
  st = cuda_check(c, cudaGetLastError(), "result copy");
  if (st != DCS_OK) return st;
  if (status & (1 << DCS_ERR_OOM)) return fail(c, DCS_ERR_OOM, "branch pool exhausted");
  if (status & (1 << DCS_ERR_UNSUPPORTED)) return fail(c, DCS_ERR_UNSUPPORTED, "branch pool above 1024 slots");
  if (status & (1 << DCS_ERR_TIMEOUT))
    return fail(c, DCS_ERR_TIMEOUT, "a bounded wait of the tensor-core pipeline gave up");
  if (status & (1 << DCS_ERR_INVALID))
    return fail(c, DCS_ERR_INVALID, "branch keep or shot fork found a list of the wrong length");
  return DCS_OK;
}

dcs_status_t dcs_get_bonds(dcs_ctx_t c, int32_t* bonds, int* n_active) {
  if (!c || !bonds) return fail(c, DCS_ERR_INVALID, "null argument");
  dcs_status_t st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronize");
  if (st != DCS_OK) return st;
  const size_t S = (size_t)c->cfg.n_slots, n1 = (size_t)c->cfg.n_qubits + 1;
  std::vector<int> cnt_v(1), order(S), kb(S), all(S * 2 * n1);
  cudaMemcpy(cnt_v.data(), c->dev.count, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(order.data(), c->dev.order, S * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(kb.data(), c->dev.ketbuf, S * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(all.data(), c->dev.bonds, all.size() * sizeof(int), cudaMemcpyDeviceToHost);
  if ((st = cuda_check(c, cudaGetLastError(), "bond copy")) != DCS_OK) return st;
  const int cnt = cnt_v[0];
  if (cnt < 0 || (size_t)cnt > S) return fail(c, DCS_ERR_CUDA, "active count out of range");
  for (int i = 0; i < cnt; ++i) {
    const int slot = order[i];
    if (slot < 0 || (size_t)slot >= S || (kb[slot] != 0 && kb[slot] != 1))
      return fail(c, DCS_ERR_CUDA, "slot list out of range");
    std::memcpy(bonds + (size_t)i * n1, all.data() + ((size_t)slot * 2 + kb[slot]) * n1,
                n1 * sizeof(int32_t));
  }
  if (n_active) *n_active = cnt;
  return DCS_OK;
}

static dcs_status_t slot_of(dcs_ctx_t c, int pos, int& slot, int& kb, std::vector<int>& bonds,
                            int& centre) {
  dcs_status_t st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronize");
  if (st != DCS_OK) return st;
  int cnt = 0;
  cudaMemcpy(&cnt, c->dev.count, sizeof(int), cudaMemcpyDeviceToHost);
  if (pos < 0 || pos >= cnt) return fail(c, DCS_ERR_INVALID, "slot is not active");
  cudaMemcpy(&slot, c->dev.order + pos, sizeof(int), cudaMemcpyDeviceToHost);
  // values read back from the device index host arrays and size host copies below: a value
  // outside its range can only come from corrupted device state and is reported
  if (slot < 0 || slot >= c->cfg.n_slots) return fail(c, DCS_ERR_CUDA, "slot list out of range");
  cudaMemcpy(&kb, c->dev.ketbuf + slot, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&centre, c->dev.centre + slot, sizeof(int), cudaMemcpyDeviceToHost);
  const int n = c->cfg.n_qubits;
  if (kb != 0 && kb != 1) return fail(c, DCS_ERR_CUDA, "buffer flag out of range");
  bonds.assign(n + 1, 0);
  cudaMemcpy(bonds.data(), c->dev.bonds + ((size_t)slot * 2 + kb) * (n + 1), (n + 1) * sizeof(int),
             cudaMemcpyDeviceToHost);
  if (st = cuda_check(c, cudaGetLastError(), "slot query"); st != DCS_OK) return st;
  if (centre < 0 || centre >= n) return fail(c, DCS_ERR_CUDA, "centre out of range");
  for (int v : bonds)
    if (v < 1 || v > c->dev.chi_cap) return fail(c, DCS_ERR_CUDA, "bond out of range");
  for (int j = 0; j <= n; ++j)
    if (bonds[j] > bond_cap(j, n, c->dev.chi_cap)) return fail(c, DCS_ERR_CUDA, "bond out of range");
  return DCS_OK;
}

dcs_status_t dcs_export_mps(dcs_ctx_t c, int pos, void* host_buf, size_t* bytes) {
  if (!c || !bytes) return fail(c, DCS_ERR_INVALID, "null argument");
  int slot, kb, centre;
  std::vector<int> b;
  dcs_status_t st = slot_of(c, pos, slot, kb, b, centre);
  if (st != DCS_OK) return st;
  const int n = c->cfg.n_qubits;
  size_t need = sizeof(int32_t) * (n + 3);
  for (int j = 0; j < n; ++j) need += sizeof(float2) * (size_t)b[j] * 2 * b[j + 1];
  if (!host_buf) {
    *bytes = need;
    return DCS_OK;
  }
  if (*bytes < need) return fail(c, DCS_ERR_INVALID, "export buffer too small");
  char* o = static_cast<char*>(host_buf);
  int32_t hdr = n;
  std::memcpy(o, &hdr, 4);
  std::memcpy(o + 4, b.data(), 4 * (n + 1));
  std::memcpy(o + 4 * (n + 2), &centre, 4);
  size_t off = 4 * (size_t)(n + 3);
  for (int j = 0; j < n; ++j) {
    const size_t len = (size_t)b[j] * 2 * b[j + 1];
    cudaMemcpy(o + off, c->dev.mps[kb] + (size_t)slot * c->dev.mps_slot_stride + c->site_off[j],
               len * sizeof(float2), cudaMemcpyDeviceToHost);
    off += len * sizeof(float2);
  }
  *bytes = need;
  return cuda_check(c, cudaGetLastError(), "export");
}

dcs_status_t dcs_import_mps(dcs_ctx_t c, int pos, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return fail(c, DCS_ERR_INVALID, "null argument");
  int slot, kb, centre_old;
  std::vector<int> bo;
  dcs_status_t st = slot_of(c, pos, slot, kb, bo, centre_old);
  if (st != DCS_OK) return st;
  const int n = c->cfg.n_qubits;
  const char* in = static_cast<const char*>(host_buf);
  if (bytes < sizeof(int32_t) * (n + 3)) return fail(c, DCS_ERR_INVALID, "import buffer too small");
  int32_t hn;
  std::memcpy(&hn, in, 4);
  if (hn != n) return fail(c, DCS_ERR_INVALID, "qubit count mismatch");
  std::vector<int> b(n + 1);
  std::memcpy(b.data(), in + 4, 4 * (n + 1));
  int32_t centre;
  std::memcpy(&centre, in + 4 * (n + 2), 4);
  if (b[0] != 1 || b[n] != 1 || centre < 0 || centre >= n)
    return fail(c, DCS_ERR_INVALID, "malformed MPS header");
  size_t need = sizeof(int32_t) * (n + 3);
  for (int j = 0; j <= n; ++j)
    if (b[j] < 1 || b[j] > bond_cap(j, n, c->dev.chi_cap))
      return fail(c, DCS_ERR_INVALID, "bond above capacity");
  for (int j = 0; j < n; ++j) need += sizeof(float2) * (size_t)b[j] * 2 * b[j + 1];
  if (bytes < need) return fail(c, DCS_ERR_INVALID, "import buffer too small");
  size_t off = 4 * (size_t)(n + 3);
  for (int j = 0; j < n; ++j) {
    const size_t len = (size_t)b[j] * 2 * b[j + 1];
    cudaMemcpy(c->dev.mps[kb] + (size_t)slot * c->dev.mps_slot_stride + c->site_off[j],
               in + off, len * sizeof(float2), cudaMemcpyHostToDevice);
    off += len * sizeof(float2);
  }
  cudaMemcpy(c->dev.bonds + ((size_t)slot * 2 + kb) * (n + 1), b.data(), (n + 1) * sizeof(int),
             cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.centre + slot, &centre, sizeof(int), cudaMemcpyHostToDevice);
  for (int j = 0; j <= n; ++j) c->ub[j] = std::max(c->ub[j], b[j]);
  // the copies above run on the default stream and may return before their DMA is done:
  // finish them before later work on the context's stream reads the slot
  return cuda_check(c, cudaDeviceSynchronize(), "import");
}

dcs_status_t dcs_branch_append(dcs_ctx_t c, const void* host_buf, size_t bytes, double p,
                               double F, const uint64_t* cwords, uint8_t flags) {
  if (!c || !host_buf || !cwords) return fail(c, DCS_ERR_INVALID, "null argument");
  if (!c->multipath) return fail(c, DCS_ERR_INVALID, "appending a branch needs multi-path mode");
  if (!(p >= 0.0) || !std::isfinite(p) || !std::isfinite(F))
    return fail(c, DCS_ERR_INVALID, "p must be finite and >= 0, F finite");
  const int n = c->cfg.n_qubits;
  const char* in = static_cast<const char*>(host_buf);
  if (bytes < sizeof(int32_t) * (n + 3)) return fail(c, DCS_ERR_INVALID, "branch buffer too small");
  int32_t hn, centre;
  std::memcpy(&hn, in, 4);
  if (hn != n) return fail(c, DCS_ERR_INVALID, "qubit count mismatch");
  std::vector<int> b(n + 1);
  std::memcpy(b.data(), in + 4, 4 * (n + 1));
  std::memcpy(&centre, in + 4 * (n + 2), 4);
  if (b[0] != 1 || b[n] != 1 || centre < 0 || centre >= n)
    return fail(c, DCS_ERR_INVALID, "malformed MPS header");
  size_t need = sizeof(int32_t) * (n + 3);
  for (int j = 0; j <= n; ++j)
    if (b[j] < 1 || b[j] > bond_cap(j, n, c->dev.chi_cap))
      return fail(c, DCS_ERR_INVALID, "bond above capacity");
  for (int j = 0; j < n; ++j) need += sizeof(float2) * (size_t)b[j] * 2 * b[j + 1];
  if (bytes < need) return fail(c, DCS_ERR_INVALID, "branch buffer too small");
  // the active list, read back after the queued work: a free slot is one not on it
  dcs_status_t st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronize");
  if (st != DCS_OK) return st;
  const int S = c->cfg.n_slots;
  int cnt = 0;
  std::vector<int> order(S);
  cudaMemcpy(&cnt, c->dev.count, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(order.data(), c->dev.order, S * sizeof(int), cudaMemcpyDeviceToHost);
  if ((st = cuda_check(c, cudaGetLastError(), "list query")) != DCS_OK) return st;
  if (cnt < 0 || cnt > S) return fail(c, DCS_ERR_CUDA, "active count out of range");
  if (cnt == S) return fail(c, DCS_ERR_OOM, "branch pool full");
  std::vector<char> used(S, 0);
  for (int i = 0; i < cnt; ++i) {
    if (order[i] < 0 || order[i] >= S) return fail(c, DCS_ERR_CUDA, "slot list out of range");
    used[order[i]] = 1;
  }
  int slot = 0;
  while (used[slot]) ++slot;
  const int kb = 0;
  size_t off = 4 * (size_t)(n + 3);
  for (int j = 0; j < n; ++j) {
    const size_t len = (size_t)b[j] * 2 * b[j + 1];
    cudaMemcpy(c->dev.mps[kb] + (size_t)slot * c->dev.mps_slot_stride + c->site_off[j], in + off,
               len * sizeof(float2), cudaMemcpyHostToDevice);
    off += len * sizeof(float2);
  }
  const uint32_t fl = flags;
  const double rr[2] = {1.0, 0.0};
  cudaMemcpy(c->dev.bonds + ((size_t)slot * 2 + kb) * (n + 1), b.data(), (n + 1) * sizeof(int),
             cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.centre + slot, &centre, sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.ketbuf + slot, &kb, sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.p + slot, &p, sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.F + slot, &F, sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.rr + 2 * (size_t)slot, rr, 2 * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.flags + slot, &fl, sizeof(uint32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.creg + (size_t)slot * DCS_CWORDS, cwords, DCS_CWORDS * sizeof(uint64_t),
             cudaMemcpyHostToDevice);
  const int cnt1 = cnt + 1;
  cudaMemcpy(c->dev.order + cnt, &slot, sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(c->dev.count, &cnt1, sizeof(int), cudaMemcpyHostToDevice);
  for (int j = 0; j <= n; ++j) c->ub[j] = std::max(c->ub[j], b[j]);
  // the copies above run on the default stream: finish them before later work on the
  // context's stream reads the branch
  return cuda_check(c, cudaDeviceSynchronize(), "branch append");
}

dcs_status_t dcs_run_circuit(dcs_ctx_t c, const dcs_op* ops, int n_ops, uint64_t meas_idx0,
                             int max_branches) {
  if (!c || (n_ops > 0 && !ops)) return fail(c, DCS_ERR_INVALID, "null argument");
  for (int i = 0; i < n_ops; ++i) {
    dcs_status_t st = check_gate(c, ops[i]);
    if (st != DCS_OK) return st;
  }
  // resets lowered, chunks and measurement runs (Sec. "Handling unitary chunks in dynamic
  // circuits", one-layer reading)
  Program P;
  if (const char* e = plan_circuit(P, c->cfg.n_qubits, c->cfg.chunk_k, ops, n_ops, meas_idx0,
                                   c->cfg.chunk_layers))
    return fail(c, DCS_ERR_INVALID, e);
  if (P.layers.size() * sizeof(DLayer) > kProgBytes / 2)
    return fail(c, DCS_ERR_OOM, "too many chunks for one call");
  return run_steps(c, P, max_branches, nullptr);
}

}  // extern "C"
