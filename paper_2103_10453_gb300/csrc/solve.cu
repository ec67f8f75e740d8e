// solve.cu -- placeholder, replaced by the generation-loop driver.
#include "plse_handle.cuh"
namespace plse { void release_solver(plse_instance *) {} }
extern "C" {
int plse_solve(plse_handle h, int, int, int64_t, uint64_t, int8_t *, int *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
int plse_solve_ex(plse_handle h, int, int, int64_t, uint64_t, void *, int8_t *, int *, plse_solve_stats *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
int plse_distances(plse_handle h, const uint8_t *, int, const uint8_t *, int, int32_t *, void *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
int plse_pop_update(plse_handle h, int, const uint8_t *, const int64_t *, int32_t *, int32_t *, void *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
int plse_matching(plse_handle h, int, const uint8_t *, const uint32_t *, uint32_t *, int32_t *, int, uint64_t, int32_t *, int32_t *, void *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
int plse_crossover(plse_handle h, int, const uint8_t *, const int32_t *, const int32_t *, int, uint64_t, uint8_t *, void *) { return h ? PLSE_ENOTSUP : PLSE_EINVAL; }
}
