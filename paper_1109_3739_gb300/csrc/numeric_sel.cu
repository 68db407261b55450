// numeric_sel.cu -- selector instantiations (values copied bit for bit, by width).
#include "numeric.cuh"

namespace hs {
bool launch_numeric_sel(int second, int vbytes, int kind, const NumArgs &a, cudaStream_t st) {
  if (second) {
    if (vbytes == 8) launch_numeric_sr<Semiring<SELECT2ND, unsigned long long>>(kind, a, st);
    else if (vbytes == 4) launch_numeric_sr<Semiring<SELECT2ND, uint32_t>>(kind, a, st);
    else launch_numeric_sr<Semiring<OR_AND, NoVal>>(kind, a, st);
  } else {
    if (vbytes == 8) launch_numeric_sr<Semiring<SELECT1ST, unsigned long long>>(kind, a, st);
    else if (vbytes == 4) launch_numeric_sr<Semiring<SELECT1ST, uint32_t>>(kind, a, st);
    else launch_numeric_sr<Semiring<OR_AND, NoVal>>(kind, a, st);
  }
  return true;
}
}  // namespace hs
