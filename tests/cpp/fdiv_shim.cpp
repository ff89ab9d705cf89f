// Host build of the convolution kernels' fast division (csrc/fdiv.h) for the CPU tests.
#include <cstdint>

#include "fdiv.h"

extern "C" {
// out[i] = n[i] / d through make_fdiv / fdiv; also returns the multiplier and shift.
void fdiv_shim(uint32_t d, const int32_t* n, int count, int32_t* out, uint32_t* m, uint32_t* s) {
  const helm::FDiv f = helm::make_fdiv(d);
  for (int i = 0; i < count; ++i) out[i] = helm::fdiv(f, n[i]);
  *m = f.m;
  *s = f.s;
}
}
