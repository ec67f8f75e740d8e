// k_ls_w1.cu -- the tabu local-search kernels (Alg. 3, Sec. 3.3; Sec. 3.7) for
// orders with n < 32 (one 32-colour word), one colour-word class per translation unit.
#include "ls_walk.cuh"

namespace plse {
template struct LSKernels<1>;
}  // namespace plse
