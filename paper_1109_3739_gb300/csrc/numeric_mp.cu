// numeric_mp.cu -- (min, +) and (or, and) instantiations of the numeric kernels.
#include "numeric.cuh"

namespace hs {
bool launch_numeric_mp(int dtype, int kind, const NumArgs &a, cudaStream_t st) {
  switch (dtype) {
    case 1: launch_numeric_sr<Semiring<MIN_PLUS, float>>(kind, a, st); return true;
    case 2: launch_numeric_sr<Semiring<MIN_PLUS, int32_t>>(kind, a, st); return true;
  }
  return false;
}
bool launch_numeric_oa(int kind, const NumArgs &a, cudaStream_t st) {
  launch_numeric_sr<Semiring<OR_AND, NoVal>>(kind, a, st);
  return true;
}
}  // namespace hs
