// k_ls_w3.cu -- the tabu local-search kernels (Alg. 3, Sec. 3.3; Sec. 3.7) for
// orders with 64 <= n < 96 (three 32-colour words), one colour-word class per translation unit.
#include "ls_walk.cuh"

namespace plse {
template struct LSKernels<3>;
}  // namespace plse
