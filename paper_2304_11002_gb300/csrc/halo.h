// Geometry of the leaf items' shared-memory mass halos (host and device; the host
// builds the tables that index into them).
#pragma once

#ifdef __CUDACC__
#define OCTO_HD __host__ __device__
#else
#define OCTO_HD
#endif

namespace octo {
namespace items {

// The mass halo of a leaf node (the node's 8^3 cells and a border of width r) is
// kept in shared memory split by cell parity: halo coordinate h in [0, 8 + 2r) per
// axis goes to parity block (hx & 1) + 2 (hy & 1) + 4 (hz & 1), position
// (hx >> 1, hy >> 1, hz >> 1) in a G^3 sub-grid (G = 4 + r) with row pitch PY and
// plane pitch PZ.  The 32 lanes of a warp hold targets of one parity class (cells
// (2i + pa, 2j + pb, 2k + pc)), so for any stencil offset their sources are
// (i + u, j + v, k + w) in one parity block: lane offsets i + PY j + PZ k.
// Far halo, float64 path (lanes i, j < 4, k < 2 of a parity class): PY = 12 and
// PZ = 16 (mod 32) make the 16 float64 loads of each half-warp hit 16 distinct bank
// pairs.  Far halo, mixed path (lanes i, j < 4 and the even k = 2 kh, kh < 2, each
// lane also holding k + 1): PY = 12 and PZ = 8 (mod 32) make the 32 float32 loads
// hit 32 distinct banks (i + 12 j + 16 kh).  The near float64 halo of the mixed path
// is dense (small radius).
struct HaloGeom {
  int r, G, PY, PZ, PQ;  // border, sub-grid extent, row pitch, plane pitch, parity block size
};

OCTO_HD inline HaloGeom far_geom(int r, bool mixed) {
  HaloGeom g;
  g.r = r;
  g.G = 4 + r;
  g.PY = 12;
  while (g.PY < g.G) g.PY += 32;
  g.PZ = mixed ? 8 : 16;
  while (g.PZ < g.G * g.PY) g.PZ += 32;
  g.PQ = g.G * g.PZ;
  return g;
}

OCTO_HD inline HaloGeom near_geom(int r) {
  HaloGeom g;
  g.r = r;
  g.G = 4 + r;
  g.PY = g.G;
  g.PZ = g.G * g.G;
  g.PQ = g.G * g.PZ;
  return g;
}

// Offset of halo position (hx, hy, hz) from the origin of the halo.
OCTO_HD inline int halo_index(const HaloGeom& g, int hx, int hy, int hz) {
  return ((hx & 1) + 2 * (hy & 1) + 4 * (hz & 1)) * g.PQ + (hx >> 1) + g.PY * (hy >> 1) + g.PZ * (hz >> 1);
}

}  // namespace items
}  // namespace octo
