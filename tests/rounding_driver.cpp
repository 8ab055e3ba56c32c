// Host driver for test_host_rounding.py: runs the exact-to-FP64 rounding code
// of the seven-digit mode product and the integer-limb band products (the
// functions of fp64_round.cuh, compiled for the host) on cases read from stdin
// and prints the bit pattern of each result.
//   "acc hh mm ll SE"                 one product
//   "pair hh mm ll SX hh mm ll SY"    two products summed exactly
//   "c7 I0 .. I6 SE"                  seven-digit recombination
#include <cstdio>
#include <cstring>

#include "fp64_round.cuh"

static void emit(double r) {
  unsigned long long b;
  std::memcpy(&b, &r, 8);
  std::printf("%llu\n", b);
}

int main() {
  char kind[8];
  while (std::scanf("%7s", kind) == 1) {
    if (!std::strcmp(kind, "acc")) {
      stfd::Acc a;
      int se;
      if (std::scanf("%lld %lld %lld %d", &a.hh, &a.mm, &a.ll, &se) != 4) return 1;
      emit(stfd::round_acc(a, se));
    } else if (!std::strcmp(kind, "pair")) {
      stfd::Acc x, y;
      int sx, sy;
      if (std::scanf("%lld %lld %lld %d %lld %lld %lld %d", &x.hh, &x.mm, &x.ll, &sx, &y.hh, &y.mm, &y.ll, &sy) != 8)
        return 1;
      emit(stfd::round_pair_exact(x, sx, y, sy));
    } else if (!std::strcmp(kind, "c7")) {
      int I[7], se;
      for (int c = 0; c < 7; ++c)
        if (std::scanf("%d", &I[c]) != 1) return 1;
      if (std::scanf("%d", &se) != 1) return 1;
      emit(stfd::combine7_int(I, se));
    } else {
      return 1;
    }
  }
  return 0;
}
