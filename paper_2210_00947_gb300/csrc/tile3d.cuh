// Geometry shared by the z-marching tiled kernels of the finest 3D level: a
// 32 x 8 block owns a column of nodes, shared memory holds the node plane
// tiles with a one-node ring and the element layer tiles with a one-element
// ring on the low side, each thread loads its own node and element, and the
// ring cells are loaded by the first three warps (planes) and warps 4-5
// (layers).
#pragma once

namespace mgar {
namespace tile {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int XS = 4, KS = 3;                  // plane and layer slots
constexpr int XRING = 2 * (TX + 2) + 2 * TY;   // 84 ring nodes of a plane tile
constexpr int KRING = (TX + 1) + TY;           // 41 ring elements of a layer tile
constexpr int KRING0 = 128;                    // first thread of the layer ring

// ring cell q of a plane tile -> halo coordinates (hx in 0..TX+1, hy in 0..TY+1)
__device__ __forceinline__ void xring(int q, int& hx, int& hy) {
  if (q < TX + 2) { hx = q; hy = 0; }
  else if (q < 2 * (TX + 2)) { hx = q - (TX + 2); hy = TY + 1; }
  else if (q < 2 * (TX + 2) + TY) { hx = 0; hy = q - 2 * (TX + 2) + 1; }
  else { hx = TX + 1; hy = q - 2 * (TX + 2) - TY + 1; }
}
// ring cell q of a layer tile -> (hx in 0..TX, hy in 0..TY)
__device__ __forceinline__ void kring(int q, int& hx, int& hy) {
  if (q < TX + 1) { hx = q; hy = 0; }
  else { hx = 0; hy = q - TX; }
}

}  // namespace tile
}  // namespace mgar
