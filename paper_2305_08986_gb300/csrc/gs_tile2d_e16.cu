// 2D cell-tile kernel (gs_tile2d.cuh), tiles of 32 x 16 evaluated cells.
#include "gs_tile2d.cuh"

namespace gs {

template <typename T>
cudaError_t launch_tile2d_e16(int mode, int ops, const TileArgs<T>& a, cudaStream_t st) {
  return tile2d::launch_shape<T, 16, true>(mode, ops, a, st);
}
template cudaError_t launch_tile2d_e16<float>(int, int, const TileArgs<float>&, cudaStream_t);
template cudaError_t launch_tile2d_e16<double>(int, int, const TileArgs<double>&, cudaStream_t);

}  // namespace gs

namespace gs {

// Variant per launch: TileArgs::shape 0 -> tiles of 16 rows of evaluated cells, 1 -> 17, 2 -> 8,
// 3 -> the strip kernel for the velocity block (gs_strip2d.cu; tiles of 8 rows for the other
// blocks).  The result does not depend on the variant: every node sums its cell contributions in
// the same fixed order.
template <typename T>
cudaError_t launch_tile2d(int mode, int ops, TileArgs<T> a, cudaStream_t st) {
  if (mode == TILE_CHEB && ops != OPS_A) return cudaErrorInvalidValue;
  // corrector stage: launches that include the velocity block take the convection terms (32 x 8
  // tiles); B and B^T alone are unchanged
  if (a.conv && (ops & OPS_A)) return launch_tile2d_conv<T>(mode, ops, a, st);
  if (a.shape == 3 && ops == OPS_A && 2 * a.g.Nv < (1LL << 31)) return launch_strip2d<T>(mode, a, st);
  if (a.shape == 1) return launch_tile2d_e17<T>(mode, ops, a, st);
  if (a.shape == 2 || a.shape == 3) return launch_tile2d_e8<T>(mode, ops, a, st);
  return launch_tile2d_e16<T>(mode, ops, a, st);
}
template cudaError_t launch_tile2d<float>(int, int, TileArgs<float>, cudaStream_t);
template cudaError_t launch_tile2d<double>(int, int, TileArgs<double>, cudaStream_t);

}  // namespace gs
