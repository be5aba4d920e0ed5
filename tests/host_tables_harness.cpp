// Host-only driver of libdcs's chunk-table builder (build_layer in dcs_tables.h) for the CPU
// tests: reads n and a file of dcs_op records (one chunk, circuit order), builds the chunk's
// tables exactly as the library does before uploading them, and prints them as text.
// No CUDA call is made; it runs without a GPU.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dcs_tables.h"

using namespace dcs;

namespace {

struct Prog {  // the containers build_layer appends to
  std::vector<DLayer> layers;
  std::vector<DBlock> blocks;
  std::vector<DGate1> g1;
  std::vector<DCond> conds;
  bool overflow() const { return false; }
};

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
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s n ops.bin\n", argv[0]);
    return 2;
  }
  const int n = std::atoi(argv[1]);
  FILE* f = std::fopen(argv[2], "rb");
  if (!f) return 2;
  std::vector<dcs_op> ops;
  dcs_op o;
  while (std::fread(&o, sizeof(o), 1, f) == 1) ops.push_back(o);
  std::fclose(f);
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
