// dcs_compress_noalloc: one compression step of one MPS that allocates no memory.
//
// The paper has no counterpart to this entry point.  It exists for callers that cannot
// allocate device memory: code that runs under a framework owning every byte of the GPU
// through its own pool, or inside a section where a cudaMalloc would synchronise the
// device or is forbidden.  The caller passes the input and output buffers; the working
// memory (environment caches, per-MPS state, the chunk's tables) lives in the file-scope
// device array below, whose size is fixed at build time.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "dcs_kernels.cuh"
#include "dcs_tables.h"

namespace {

using namespace dcs;

// Working memory of dcs_compress_noalloc.  Every GPU that loads the library holds it until
// the process exits.  All calls share it, and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DCS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
std::mutex g_mu;                    // guards g_scratch_addr and the host table staging

template <class T, int N>
struct FixedVec {
  T v[N];
  int n = 0;
  bool over = false;
  void push_back(const T& x) {
    if (n < N) v[n++] = x;
    else over = true;
  }
  int size() const { return n; }
  const T* data() const { return v; }
};

// Host staging of one chunk's tables (static storage: no heap use per call).
struct FixedProg {
  FixedVec<DLayer, 1> layers;
  FixedVec<DBlock, DCS_NOALLOC_MAX_QUBITS / 2> blocks;
  FixedVec<DGate1, DCS_NOALLOC_MAX_GATES> g1;
  FixedVec<DCond, DCS_NOALLOC_MAX_GATES> conds;
  bool overflow() const { return layers.over || blocks.over || g1.over || conds.over; }
  void clear() {
    layers.n = blocks.n = g1.n = conds.n = 0;
    layers.over = blocks.over = g1.over = conds.over = false;
  }
};
FixedProg g_prog;

size_t up(size_t x) { return (x + 255) / 256 * 256; }

struct Carve {
  size_t mps, env, offs, bonds, ints, dbl, creg, flags, shot, plan, layer, blocks, g1, conds, total;
};

Carve carve(int n, int C) {
  Carve k{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o = up(o + b);
    return r;
  };
  const size_t env = (size_t)(n + 1) * 4 * C * C * sizeof(float2);
  k.mps = take((size_t)n * 2 * C * C * sizeof(float2));  // the second MPS buffer
  k.env = take(env);
  k.offs = take(2 * (size_t)(n + 1) * sizeof(size_t));
  k.bonds = take(2 * (size_t)(n + 1) * sizeof(int32_t));
  k.ints = take(8 * sizeof(int32_t));   // centre, ketbuf, order, count, status
  k.dbl = take(4 * sizeof(double));     // p, F, rr[2]
  k.creg = take(DCS_CWORDS * sizeof(uint64_t));
  k.flags = take(sizeof(uint32_t));
  k.shot = take(sizeof(uint64_t));
  k.plan = take((PLAN_HDR + 4) * sizeof(int32_t));
  k.layer = take(sizeof(DLayer));
  k.blocks = take(sizeof(DBlock) * (DCS_NOALLOC_MAX_QUBITS / 2));
  k.g1 = take(sizeof(DGate1) * DCS_NOALLOC_MAX_GATES);
  k.conds = take(sizeof(DCond) * DCS_NOALLOC_MAX_GATES);
  k.total = o;
  return k;
}

struct Creg {
  uint64_t w[DCS_CWORDS];
};

// Per-call state of the single slot: nothing carries over from the previous call.  The
// caller's ket is read only: it is copied into the caller's bra buffer, which serves as the
// slot's first MPS buffer (an exact step updates it in place; otherwise the result lands in
// the scratch MPS buffer and k_noalloc_finish copies it over).
//
// The caller's bonds are checked here, on the device, before any kernel indexes with them:
// bond 0 and bond n must be 1 and every bond must lie in 1 .. C (the site stride holds
// C x 2 x C).  A malformed list leaves the active count at 0, so the compression kernel
// returns at once, and k_noalloc_finish reports the failure.
__global__ void k_noalloc_prepare(DevCtx c, const int32_t* ket_bonds, int centre, Creg creg,
                                  const float2* ket) {
  const int n = c.n, C = c.chi_cap;
  const size_t stride = 2 * (size_t)C * C;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = (ket_bonds[0] != 1 || ket_bonds[n] != 1) ? 1 : 0;
  __syncthreads();
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    const int b = ket_bonds[i];
    if (b < 1 || b > C) atomicOr(&bad, 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    const int b = bad ? 1 : ket_bonds[i];
    c.bonds[i] = b;
    c.bonds[n + 1 + i] = b;
    const_cast<size_t*>(c.site_off)[i] = (size_t)i * stride;
    const_cast<size_t*>(c.env_off)[i] = (size_t)i * 2 * stride;
  }
  for (int j = 0; j < n && !bad; ++j) {
    const int len = ket_bonds[j] * 2 * ket_bonds[j + 1];
    for (int e = threadIdx.x; e < len; e += blockDim.x)
      c.mps[0][(size_t)j * stride + e] = ket[(size_t)j * stride + e];
  }
  if (threadIdx.x < DCS_CWORDS) c.creg[threadIdx.x] = creg.w[threadIdx.x];
  if (threadIdx.x == 0) {
    c.order[0] = 0;
    *c.count = bad ? 0 : 1;
    *c.status = 0;
    c.centre[0] = centre;
    c.ketbuf[0] = 0;
    c.p[0] = 1.0;
    c.F[0] = 1.0;
    c.rr[0] = 1.0;
    c.rr[1] = 0.0;
    c.flags[0] = 0u;
    c.shot[0] = 0ull;
  }
}

// Bond dimensions and centre of the result.  The bra buffer already holds it unless the
// step swapped buffers (the sweeps ran): then it is copied over from the scratch buffer.  A
// slot left unchanged (every gate skipped by its condition) hands back the input; an empty
// chunk sets f = 1 here.  Failures become visible in the outputs: malformed ket bonds give
// bra_bonds[0] = 0, bra_centre = -1 and f = NaN; a NaN/Inf met in the step, or a bounded
// device wait that gave up, gives f = NaN.
__global__ void k_noalloc_finish(DevCtx c, int32_t* bra_bonds, int32_t* bra_centre,
                                 float2* bra, double* f, int empty) {
  const int n = c.n;
  const size_t stride = 2 * (size_t)c.chi_cap * c.chi_cap;
  if (*c.count == 0) {
    if (threadIdx.x == 0) {
      bra_bonds[0] = 0;
      if (bra_centre) *bra_centre = -1;
      *f = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const int buf = c.ketbuf[0];
  const int* bd = c.bonds + buf * (n + 1);
  for (int i = threadIdx.x; i <= n; i += blockDim.x) bra_bonds[i] = bd[i];
  if (buf == 1) {
    for (int j = 0; j < n; ++j) {
      const int len = bd[j] * 2 * bd[j + 1];
      for (int e = threadIdx.x; e < len; e += blockDim.x)
        bra[(size_t)j * stride + e] = c.mps[1][(size_t)j * stride + e];
    }
  }
  if (threadIdx.x == 0) {
    if (bra_centre) *bra_centre = c.centre[0];
    if (empty) *f = 1.0;
    if ((c.flags[0] & DCS_FLAG_NUMERICAL) || *c.status != 0)
      *f = __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

extern "C" dcs_status_t dcs_compress_noalloc(int32_t n_qubits, int32_t chi_max, double tol,
                                            int32_t sweeps, const dcs_op* gates,
                                            int32_t n_gates, const uint64_t* creg,
                                            const void* ket, const int32_t* ket_bonds,
                                            int32_t ket_centre, void* bra, int32_t* bra_bonds,
                                            int32_t* bra_centre, double* f,
                                            dcs_stream_t stream) {
  if (n_qubits < 1 || chi_max < 1 || sweeps < 1 || !(tol >= 0.0) || n_gates < 0 ||
      (n_gates > 0 && !gates) || !ket || !ket_bonds || !bra || !bra_bonds || !f ||
      ket_centre < 0 || ket_centre >= n_qubits)
    return DCS_ERR_INVALID;
  if (n_qubits > DCS_NOALLOC_MAX_QUBITS || chi_max > DCS_NOALLOC_MAX_CHI ||
      n_gates > DCS_NOALLOC_MAX_GATES)
    return DCS_ERR_OOM;  // beyond what the fixed scratch holds
  for (int i = 0; i < n_gates; ++i) {
    const dcs_op& o = gates[i];
    if (o.kind != DCS_OP_GATE1 && o.kind != DCS_OP_GATE2) return DCS_ERR_INVALID;
    const bool two = o.kind == DCS_OP_GATE2;
    if (o.q0 < 0 || o.q0 >= n_qubits || (two && (o.q1 < 0 || o.q1 >= n_qubits)))
      return DCS_ERR_INVALID;
    if (!cond_valid(o.cond))
      return DCS_ERR_INVALID;
  }
  const int C = fused_chi(chi_max);
  const Carve k = carve(n_qubits, C);
  if (k.total > DCS_NOALLOC_SCRATCH_BYTES) return DCS_ERR_OOM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DCS_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    // Once per device, with that device current.  In host code g_noalloc_scratch names a
    // host-side stand-in, not device memory: only this address may be handed to kernels.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DCS_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  char* base = static_cast<char*>(g_scratch_addr[dev]);

  g_prog.clear();
  if (n_gates > 0 && build_layer(g_prog, n_qubits, gates, n_gates) != nullptr) return DCS_ERR_INVALID;

  DevCtx d{};
  d.n = n_qubits;
  d.chi_cap = C;
  d.dmax = 4;
  d.n_slots = 1;
  d.mps_slot_stride = (size_t)n_qubits * 2 * C * C;
  d.env_slot_stride = (size_t)(n_qubits + 1) * 4 * C * C;
  d.mps[0] = static_cast<float2*>(bra);
  d.mps[1] = reinterpret_cast<float2*>(base + k.mps);
  d.env = reinterpret_cast<float2*>(base + k.env);
  d.site_off = reinterpret_cast<const size_t*>(base + k.offs);
  d.env_off = d.site_off + (n_qubits + 1);
  d.bonds = reinterpret_cast<int32_t*>(base + k.bonds);
  int32_t* ints = reinterpret_cast<int32_t*>(base + k.ints);
  d.centre = ints + 0;
  d.ketbuf = ints + 1;
  d.order = ints + 2;
  d.count = ints + 3;
  d.status = ints + 4;
  double* dbl = reinterpret_cast<double*>(base + k.dbl);
  d.p = dbl + 0;
  d.F = dbl + 1;
  d.rr = dbl + 2;
  d.creg = reinterpret_cast<uint64_t*>(base + k.creg);
  d.flags = reinterpret_cast<uint32_t*>(base + k.flags);
  d.shot = reinterpret_cast<uint64_t*>(base + k.shot);
  d.plan = reinterpret_cast<int32_t*>(base + k.plan);
  d.seed = 0;
  d.chi_max = chi_max;
  d.tol = tol;
  d.sweeps = sweeps;

  Creg cr{};
  if (creg) std::memcpy(cr.w, creg, sizeof(cr.w));
  k_noalloc_prepare<<<1, 128, 0, s>>>(d, ket_bonds, ket_centre, cr, static_cast<const float2*>(ket));
  if (cudaGetLastError() != cudaSuccess) return DCS_ERR_CUDA;
  if (n_gates > 0) {
    // the tables travel from static host storage; a copy from pageable memory returns once
    // the source has been staged, so g_prog may be reused by the next call
    DLayer* dl = reinterpret_cast<DLayer*>(base + k.layer);
    DBlock* db = reinterpret_cast<DBlock*>(base + k.blocks);
    DGate1* dg = reinterpret_cast<DGate1*>(base + k.g1);
    DCond* dc = reinterpret_cast<DCond*>(base + k.conds);
    if (cudaMemcpyAsync(dl, g_prog.layers.data(), sizeof(DLayer), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (g_prog.blocks.size() &&
         cudaMemcpyAsync(db, g_prog.blocks.data(), sizeof(DBlock) * g_prog.blocks.size(),
                         cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        (g_prog.g1.size() &&
         cudaMemcpyAsync(dg, g_prog.g1.data(), sizeof(DGate1) * g_prog.g1.size(),
                         cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        (g_prog.conds.size() &&
         cudaMemcpyAsync(dc, g_prog.conds.data(), sizeof(DCond) * g_prog.conds.size(),
                         cudaMemcpyHostToDevice, s) != cudaSuccess))
      return DCS_ERR_CUDA;
    launch_compress(d, C, dl, 1, db, dg, dc, f, s);
    if (cudaGetLastError() != cudaSuccess) return DCS_ERR_CUDA;
  }
  // an empty chunk has nothing to compress: k_noalloc_finish writes f = 1
  k_noalloc_finish<<<1, 128, 0, s>>>(d, bra_bonds, bra_centre, static_cast<float2*>(bra), f,
                                     n_gates == 0 ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess) return DCS_ERR_CUDA;
  return DCS_OK;
}
