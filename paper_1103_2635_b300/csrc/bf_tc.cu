// tcgen05 tensor-core BF kernel (placeholder until the kernel lands).
#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

bool tc_available() { return false; }

int launch_bf_tc_topc(const LpMatrix&, const LpMatrix&, int, const TileWork&, const TopOut&, int,
                      cudaStream_t, uint32_t*) {
  set_error("tensor-core BF kernel not built");
  return RBC_ERR_UNSUPPORTED;
}

}  // namespace rbc
