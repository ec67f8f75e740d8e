// k_ls_w4.cu -- the tabu local-search kernels (Alg. 3, Sec. 3.3; Sec. 3.7) for
// orders with 96 <= n <= 127 (four 32-colour words), one colour-word class per translation unit.
#include "ls_walk.cuh"

namespace plse {
template struct LSKernels<4>;
}  // namespace plse
