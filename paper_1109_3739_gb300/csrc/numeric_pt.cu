// numeric_pt.cu -- (+, x) instantiations of the numeric kernels.
#include "numeric.cuh"

namespace hs {
bool launch_numeric_pt(int dtype, int kind, const NumArgs &a, cudaStream_t st) {
  switch (dtype) {
    case 0: launch_numeric_sr<Semiring<PLUS_TIMES, double>>(kind, a, st); return true;
    case 1: launch_numeric_sr<Semiring<PLUS_TIMES, float>>(kind, a, st); return true;
    case 3: launch_numeric_sr<Semiring<PLUS_TIMES, int64_t>>(kind, a, st); return true;
  }
  return false;
}
}  // namespace hs
