// 2D cell-tile kernel (gs_tile2d.cuh), tiles of 32 x 8 evaluated cells.
#include "gs_tile2d.cuh"

namespace gs {

template <typename T>
cudaError_t launch_tile2d_e8(int mode, int ops, const TileArgs<T>& a, cudaStream_t st) {
  return tile2d::launch_shape<T, 8, true>(mode, ops, a, st);
}
template cudaError_t launch_tile2d_e8<float>(int, int, const TileArgs<float>&, cudaStream_t);
template cudaError_t launch_tile2d_e8<double>(int, int, const TileArgs<double>&, cudaStream_t);

template <typename T>
cudaError_t launch_tile2d_conv(int mode, int ops, const TileArgs<T>& a, cudaStream_t st) {
  return tile2d::launch_conv_shape<T, 8>(mode, ops, a, st);
}
template cudaError_t launch_tile2d_conv<float>(int, int, const TileArgs<float>&, cudaStream_t);
template cudaError_t launch_tile2d_conv<double>(int, int, const TileArgs<double>&, cudaStream_t);

}  // namespace gs
