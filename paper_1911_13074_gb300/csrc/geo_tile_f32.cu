// Kernel instantiations for f32 images: the shared-memory tile kernel and the
// register-resident kernel.
#include "geo_launch.cuh"

namespace geo {

int launch_tile_f32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem) {
  return launch_tile_impl<EF32>(L, op, conn, s, grid, smem);
}

int occupancy_tile_f32(int op, int conn, size_t smem, int *bps) { return occupancy_impl<EF32>(op, conn, smem, bps); }

int launch_rr_f32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, int variant) {
  if (variant == 1) return launch_rr_f32_v1(L, op, conn, s, grid);
  if (variant == 2) return launch_rr_f32_v2(L, op, conn, s, grid);
  return launch_rr_impl<SF32, true>(L, op, conn, s, grid);  // with the tagged form for rank codes
}

int occupancy_rr_f32(int op, int conn, int *bps, int variant) {
  if (variant == 1) return occupancy_rr_f32_v1(op, conn, bps);
  if (variant == 2) return occupancy_rr_f32_v2(op, conn, bps);
  return occupancy_rr_impl<SF32>(op, conn, bps);
}

}  // namespace geo
