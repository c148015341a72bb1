// Register-resident kernel for float32 images in shape variant 1 (band
// shape and block size in geo_common.cuh), chosen by the autotuner; its own
// translation unit so that the build compiles the variants in parallel.
#include "geo_launch.cuh"

namespace geo {

int launch_rr_f32_v1(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid) {
  return launch_rr_impl<SF32V1>(L, op, conn, s, grid);
}

int occupancy_rr_f32_v1(int op, int conn, int *bps) { return occupancy_rr_impl<SF32V1>(op, conn, bps); }

}  // namespace geo
