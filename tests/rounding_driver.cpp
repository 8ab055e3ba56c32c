// Host driver for test_host_rounding.py: runs the exact-to-FP64 rounding code
// of the seven-digit mode product and the integer-limb band products (the
// functions of fp64_round.cuh, compiled for the host) on cases read from stdin
// and prints the bit pattern of each result.
//   "acc hh mm ll SE"                 one product
//   "pair hh mm ll SX hh mm ll SY"    two products summed exactly
//   "c7 I0 .. I6 SE"                  seven-digit recombination
//   "bl bits E"                       balanced limbs of an FP64 entry (prints "h l")
//   "stw SE n C1 U1 .. Cn Un"         a stencil row sum of n 53-bit products
//   "stp SX n C.. U.. SY n C.. U.."   two stencil row sums summed exactly
#include <cstdio>
#include <cstring>

#include "fp64_round.cuh"

static void emit(double r) {
  unsigned long long b;
  std::memcpy(&b, &r, 8);
  std::printf("%llu\n", b);
}

static bool read_row(stfd::AccW& a) {
  int n;
  if (std::scanf("%d", &n) != 1) return false;
  a = stfd::AccW{0, 0, 0ull};
  for (int k = 0; k < n; ++k) {
    long long C, U;
    if (std::scanf("%lld %lld", &C, &U) != 2) return false;
    const int2 c = stfd::split_balanced(C), u = stfd::split_balanced(U);
    stfd::tapw(a, c, c.x + c.y, u);
  }
  return true;
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
    } else if (!std::strcmp(kind, "bl")) {
      unsigned long long bits;
      int E;
      if (std::scanf("%llu %d", &bits, &E) != 2) return 1;
      const int2 hl = stfd::balanced_limbs(bits, E);
      std::printf("%d %d\n", hl.x, hl.y);
    } else if (!std::strcmp(kind, "stw")) {
      int se;
      stfd::AccW a;
      if (std::scanf("%d", &se) != 1 || !read_row(a)) return 1;
      emit(stfd::round_acc(stfd::as_acc(a), se));
    } else if (!std::strcmp(kind, "stp")) {
      int sx, sy;
      stfd::AccW x, y;
      if (std::scanf("%d", &sx) != 1 || !read_row(x) || std::scanf("%d", &sy) != 1 || !read_row(y)) return 1;
      emit(stfd::round_pair_exact(stfd::as_acc(x), sx, stfd::as_acc(y), sy));
    } else {
      return 1;
    }
  }
  return 0;
}
