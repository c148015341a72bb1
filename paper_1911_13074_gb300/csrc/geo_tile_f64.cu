// Kernel instantiations for f64 images: the shared-memory tile kernel and the
// register-resident kernel.
#include "geo_launch.cuh"

namespace geo {

int launch_tile_f64(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem) {
  return launch_tile_impl<EF64>(L, op, conn, s, grid, smem);
}

int occupancy_tile_f64(int op, int conn, size_t smem, int *bps) { return occupancy_impl<EF64>(op, conn, smem, bps); }

int launch_rr_f64(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid) {
  return launch_rr_impl<SF64>(L, op, conn, s, grid);
}

int occupancy_rr_f64(int op, int conn, int *bps) { return occupancy_rr_impl<SF64>(op, conn, bps); }

}  // namespace geo
