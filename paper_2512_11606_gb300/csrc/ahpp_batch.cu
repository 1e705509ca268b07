// The batched kernel at its two tile widths.  ahpp_batch_kernel.cuh holds
// the kernel body; it is compiled once per width (16 and 32 queries per
// tile), each in a namespace of its own with its own kTile, and the entry
// points below pick the instance of a launch's tile width.
#include <algorithm>

#define AHPP_BT 32
#define AHPP_BT_NS tw32
#include "ahpp_batch_kernel.cuh"
#undef AHPP_BT
#undef AHPP_BT_NS

#define AHPP_BT 16
#define AHPP_BT_NS tw16
#include "ahpp_batch_kernel.cuh"
#undef AHPP_BT
#undef AHPP_BT_NS

namespace ahpp {

int launch_batch(const DevGraph& g, const BatchState& s, const BatchParams& p, bool bf16, int grid,
                 cudaStream_t stream) {
  return p.tile == 16 ? tw16::launch_batch(g, s, p, bf16, grid, stream)
                      : tw32::launch_batch(g, s, p, bf16, grid, stream);
}

int launch_serve_step(const DevGraph& g, const BatchParams& p, const ServeParams& sv, bool bf16, int grid,
                      cudaStream_t stream) {
  return tw32::launch_serve_step(g, p, sv, bf16, grid, stream);
}

int batch_max_grid(bool bf16, int sm_count) {
  const int a = tw32::batch_max_grid(bf16, sm_count), b = tw16::batch_max_grid(bf16, sm_count);
  return (a <= 0 || b <= 0) ? -1 : std::min(a, b);
}

}  // namespace ahpp
