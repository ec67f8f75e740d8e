// k_ls_w2.cu -- the tabu local-search kernels (Alg. 3, Sec. 3.3; Sec. 3.7) for
// orders with 32 <= n < 64 (two 32-colour words), one colour-word class per translation unit.
#include "ls_walk.cuh"

namespace plse {
template struct LSKernels<2>;
}  // namespace plse
