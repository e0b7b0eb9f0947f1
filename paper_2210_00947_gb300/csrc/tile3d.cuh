// Geometry of the z-marching tiled kernels of the finest 3D level: a block
// of TX x TY threads owns a TX x TY column of nodes; shared memory holds the
// node plane tiles with a one-node ring and the element layer tiles with a
// one-element ring on the low side.  Each thread loads its own node and
// element; the ring cells are loaded by the first warps (planes, XRING
// threads) and by the next warps (layers, KRING threads from KRING0).
//
// The tile width need not be a multiple of 32 (warps then span two rows):
// the df64 operator picks, per grid, the shape with the fewest idle lanes,
// e.g. 43 x 11 for 129 x 129 node planes (3 x 12 tiles, 96 % of the lanes
// busy) instead of 32 x 8 (5 x 17 tiles, 77 %); the FP32 kernels, which
// keep four blocks per SM, take 43 x 5 (3 x 26 tiles of 7 warps, 95 %).
#pragma once

namespace mgar {
namespace tile {

template <int TX_, int TY_>
struct Tile {
  static constexpr int TX = TX_, TY = TY_, NT = TX * TY;
  static constexpr int NTB = (NT + 31) / 32 * 32;          // threads launched (whole warps)
  static constexpr int XRING = 2 * (TX + 2) + 2 * TY;      // ring nodes of a plane tile
  static constexpr int KRING = (TX + 1) + TY;              // ring elements of a layer tile
  static constexpr int KRING0 = (XRING + 31) / 32 * 32;    // first thread of the layer ring
  static_assert(KRING0 + KRING <= NT, "the ring loads need more threads");

  // ring cell q of a plane tile -> halo coordinates (hx in 0..TX+1, hy in 0..TY+1)
  __device__ static __forceinline__ void xring(int q, int& hx, int& hy) {
    if (q < TX + 2) { hx = q; hy = 0; }
    else if (q < 2 * (TX + 2)) { hx = q - (TX + 2); hy = TY + 1; }
    else if (q < 2 * (TX + 2) + TY) { hx = 0; hy = q - 2 * (TX + 2) + 1; }
    else { hx = TX + 1; hy = q - 2 * (TX + 2) - TY + 1; }
  }
  // ring cell q of a layer tile -> (hx in 0..TX, hy in 0..TY)
  __device__ static __forceinline__ void kring(int q, int& hx, int& hy) {
    if (q < TX + 1) { hx = q; hy = 0; }
    else { hx = 0; hy = q - TX; }
  }
};

using T32x8 = Tile<32, 8>;
using T43x11 = Tile<43, 11>;
using T43x5 = Tile<43, 5>;

// Fraction of busy lanes of a TX x TY tiling of an NX x NY node plane.
inline double tile_use(int NX, int NY, int TX, int TY) {
  const int gx = (NX + TX - 1) / TX, gy = (NY + TY - 1) / TY;
  const int nt = TX * TY, warps = (nt + 31) / 32;
  return (double)NX * NY / ((double)gx * TX * gy * TY) * (double)nt / (32.0 * warps);
}

}  // namespace tile
}  // namespace mgar
