// Navigation of the octree of Sec. 3.3 Step 1 in its device layout: boxes of
// one level are stored contiguously, sorted by their Morton key (x bit above
// y bit above z bit at every depth), so a box is found from its integer
// coordinates by a binary search of the level's keys.  Shared by the tree
// builder and the off-surface field evaluation.
#pragma once

#include <math.h>
#include <stdint.h>

// interleave the low 21 bits of v with two zero bits between each
__device__ __host__ inline uint64_t spread3h(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// global index of the box with coordinates (x, y, z) at `level` among the
// level's nbox boxes starting at box0 of the key array, or -1 if there is none
__device__ inline int find_box_at(const uint64_t *bkey, int box0, int nbox, int level, int x, int y, int z)
{
    const int side = 1 << level;
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
    const uint64_t key = (spread3h((uint64_t)x) << 2) | (spread3h((uint64_t)y) << 1) | spread3h((uint64_t)z);
    int lo = box0, hi = box0 + nbox - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const uint64_t k = bkey[mid];
        if (k == key) return mid;
        if (k < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// cone index of direction (dx, dy, dz) at a high-frequency level with nc x nc
// cells per cube face: face (2 axis + sign) of the largest component, then
// the cell of the other two components divided by it
__device__ __host__ inline int cone_index(double dx, double dy, double dz, int nc)
{
    double d[3] = {dx, dy, dz};
    double ad[3] = {fabs(dx), fabs(dy), fabs(dz)};
    int ax = 0;
    if (ad[1] > ad[ax]) ax = 1;
    if (ad[2] > ad[ax]) ax = 2;
    int s = d[ax] > 0 ? 1 : 0;
    int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
    double u = d[o0] / ad[ax], v = d[o1] / ad[ax];
    int a = (int)floor((u + 1.0) * 0.5 * nc), b = (int)floor((v + 1.0) * 0.5 * nc);
    a = a < 0 ? 0 : (a > nc - 1 ? nc - 1 : a);
    b = b < 0 ? 0 : (b > nc - 1 ? nc - 1 : b);
    return (2 * ax + s) * nc * nc + a * nc + b;
}
