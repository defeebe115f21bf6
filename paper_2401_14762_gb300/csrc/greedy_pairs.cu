// Instances of the greedy kernel for complex data on the real form: each complex atom is
// the column pair (2j, 2j + 1), selected and pruned by its modulus (see greedy.cu).
#include "greedy_kernel.cuh"

namespace cs {

const void* greedy_pairs_kernel(int algo, int vr) {
  if (algo == kGomp) return reinterpret_cast<const void*>(greedy_kernel<kGomp, true>(vr));
  if (algo == kBiht) return reinterpret_cast<const void*>(greedy_kernel<kBiht, true>(vr));
  return reinterpret_cast<const void*>(greedy_kernel<kCosamp, true>(vr));
}

}  // namespace cs
