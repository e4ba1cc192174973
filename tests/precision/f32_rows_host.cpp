// Test harness: the float path's per-argument code (boys_f32_row.cuh, which
// compiles for the host as well) evaluated on the CPU.  The host's sqrt and
// division are correctly rounded where the GPU uses its approximate
// reciprocal square root and fast division, so this checks the arithmetic
// scheme (float-float steps, compensated chain), not the device's bits.
//   f32_rows_host <n_max> <0: closed form | 1: asymptote> <x.bin> <out.bin>
// x.bin: float32 arguments; out.bin: float32 rows [count, n_max + 1].
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "boys_f32_row.cuh"

static const float kTab[64] = BOYS_EXP2_FRAC32_FF;

template <int NMAX>
static void rows(const std::vector<float> &x, std::vector<float> &out, int mode) {
  constexpr int NTOP = NMAX <= 8 ? NMAX : NMAX + 1;  // the float path's evaluated order
  out.resize(x.size() * (NMAX + 1));
  for (size_t i = 0; i < x.size(); ++i) {
    float F[NMAX + 1];
    if (mode == 0) boys::f32_formula<NTOP, NMAX>(x[i], F, kTab);
    else boys::f32_asymptote<NMAX>(x[i], F);
    for (int m = 0; m <= NMAX; ++m) out[i * (NMAX + 1) + m] = F[m];
  }
}

int main(int argc, char **argv) {
  if (argc != 5) return 2;
  const int n_max = atoi(argv[1]), mode = atoi(argv[2]);
  FILE *f = fopen(argv[3], "rb");
  if (!f) return 3;
  fseek(f, 0, SEEK_END);
  const long bytes = ftell(f);
  fseek(f, 0, SEEK_SET);
  std::vector<float> x(bytes / 4);
  if (fread(x.data(), 4, x.size(), f) != x.size()) return 4;
  fclose(f);
  std::vector<float> out;
  switch (n_max) {
    case 8: rows<8>(x, out, mode); break;
    case 16: rows<16>(x, out, mode); break;
    case 17: rows<17>(x, out, mode); break;
    case 24: rows<24>(x, out, mode); break;
    case 36: rows<36>(x, out, mode); break;
    default: return 5;
  }
  FILE *o = fopen(argv[4], "wb");
  if (!o) return 6;
  fwrite(out.data(), 4, out.size(), o);
  fclose(o);
  return 0;
}
