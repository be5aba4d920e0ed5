// Host-only driver of libdcs's table builder and circuit planner for the CPU tests.
//   harness n ops.bin                      one chunk (dcs_op records, circuit order) through
//                                          build_layer (dcs_tables.h): its tables as text
//   harness plan n chunk_k idx0 ops.bin [layers]
//                                          a whole circuit through plan_circuit
//                                          (dcs_plan.h): steps, chunks (one CHUNK line per
//                                          sub-layer) and measurements
// No CUDA call is made; it runs without a GPU.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dcs_plan.h"

using namespace dcs;

namespace {

struct Prog {  // the containers build_layer and plan_circuit append to
  std::vector<DLayer> layers;
  std::vector<DBlock> blocks;
  std::vector<DGate1> g1;
  std::vector<DCond> conds;
  std::vector<DMeas> meas;
  std::vector<Step> steps;
  bool overflow() const { return false; }
};

std::vector<dcs_op> read_ops(const char* path) {
  std::vector<dcs_op> ops;
  FILE* f = std::fopen(path, "rb");
  if (!f) return ops;
  dcs_op o;
  while (std::fread(&o, sizeof(o), 1, f) == 1) ops.push_back(o);
  std::fclose(f);
  return ops;
}

int plan_main(int n, int chunk_k, unsigned long long idx0, const char* path, int layers) {
  std::vector<dcs_op> ops = read_ops(path);
  Prog P;
  const char* e = plan_circuit(P, n, chunk_k, ops.data(), (int)ops.size(), idx0, layers);
  if (e) {
    std::printf("ERR %s\n", e);
    return 0;
  }
  for (const Step& st : P.steps) {
    std::printf("STEP %d %d %d\n", st.kind, st.idx, st.n);
    if (st.kind == 0) {
      for (int l = 0; l < st.n; ++l) {
        const DLayer& L = P.layers[st.idx + l];
        std::printf("CHUNK %d %d %d", L.n_blocks, L.uncond, L.n_conds);
        for (int j = 0; j < n; ++j) std::printf(" %d", L.site[j].kind);
        std::printf("\n");
      }
    } else {
      for (int i = 0; i < st.n; ++i) {
        const DMeas& m = P.meas[st.idx + i];
        std::printf("MEAS %d %d %llu\n", m.q, m.cbit, (unsigned long long)m.ordinal);
      }
    }
  }
  return 0;
}

void put_c16(const char* tag, const float2* a) {
  std::printf("%s", tag);
  for (int i = 0; i < 16; ++i) std::printf(" %.9g %.9g", a[i].x, a[i].y);
  std::printf("\n");
}

void put_cond(const DCond& c) {
  std::printf(" %d %d", c.op, c.value);
  for (int w = 0; w < DCS_CWORDS; ++w) std::printf(" %llu", (unsigned long long)c.mask[w]);
}

}  // namespace

int main(int argc, char** argv) {
  if ((argc == 6 || argc == 7) && std::strcmp(argv[1], "plan") == 0)
    return plan_main(std::atoi(argv[2]), std::atoi(argv[3]), std::strtoull(argv[4], nullptr, 10),
                     argv[5], argc == 7 ? std::atoi(argv[6]) : 1);
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s n ops.bin | %s plan n chunk_k idx0 ops.bin\n", argv[0],
                 argv[0]);
    return 2;
  }
  const int n = std::atoi(argv[1]);
  std::vector<dcs_op> ops = read_ops(argv[2]);
  Prog P;
  const char* e = build_layer(P, n, ops.data(), (int)ops.size());
  if (e) {
    std::printf("ERR %s\n", e);
    return 0;
  }
  const DLayer& L = P.layers[0];
  std::printf("LAYER %d %d %d %d %d\n", L.n_blocks, L.blk_off, L.uncond, L.cond_off, L.n_conds);
  for (int j = 0; j < n; ++j)
    std::printf("SITE %d %d %d %d %d\n", j, L.site[j].kind, L.site[j].blk, L.site[j].g_off,
                L.site[j].g_n);
  for (size_t b = 0; b < P.blocks.size(); ++b) {
    const DBlock& B = P.blocks[b];
    std::printf("BLOCK %d %d %d", B.q, B.D, B.composed);
    for (int s = 0; s < 2; ++s)
      std::printf(" %d %d %d %d", B.pre_off[s], B.pre_n[s], B.post_off[s], B.post_n[s]);
    put_cond(B.cond);
    std::printf("\n");
    put_c16("G", B.G);
    put_c16("WL", B.WL);
    put_c16("WR", B.WR);
    put_c16("GC", B.Gc);
  }
  for (size_t i = 0; i < P.g1.size(); ++i) {
    std::printf("G1");
    for (int k = 0; k < 4; ++k) std::printf(" %.9g %.9g", P.g1[i].u[k].x, P.g1[i].u[k].y);
    put_cond(P.g1[i].cond);
    std::printf("\n");
  }
  for (size_t i = 0; i < P.conds.size(); ++i) {
    std::printf("COND");
    put_cond(P.conds[i]);
    std::printf("\n");
  }
  return 0;
}
