// Internal helpers shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "rsdft.h"

namespace rs {

// Per-thread last-error message (rs_last_error).
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);

}  // namespace rs

// Host-side grid: integer lattice points of a union of spheres or a box.
struct rs_grid {
    int64_t npts = 0;
    int32_t origin[3] = {0, 0, 0};   // lattice coordinate of map element (0,0,0)
    int32_t dims[3] = {0, 0, 0};     // map extents (bounding box + 4-point margin)
    double h = 0.0;
    int order = 4;                   // point order: brick edge (1, 2, 4, 8), RS_ORDER_MORTON or RS_ORDER_TILECOL
    double center[3] = {0.0, 0.0, 0.0};  // coords = (ijk - center) * h
    std::vector<int32_t> ijk;        // [npts][3]
    std::vector<int32_t> map;        // [dims0][dims1][dims2], -1 = not a grid point

    double coord(int axis, int32_t i) const { return ((double)i - center[axis]) * h; }
    int64_t map_size() const { return (int64_t)dims[0] * dims[1] * dims[2]; }
};

// Host-side Kleinman-Bylander projector tables (atom-major sphere lists).
struct rs_proj {
    int32_t n_atoms = 0;
    std::vector<int64_t> off;     // [n_atoms+1]
    std::vector<int32_t> idx;     // [n_entries] point ids, ascending per atom
    std::vector<double> gam;      // [n_entries][4]
    std::vector<double> E;        // [n_atoms][4] couplings per projector (s, p, p, p)
};

#define RS_TRY(expr)                                     \
    do {                                                 \
        int rs_try_rc_ = (expr);                         \
        if (rs_try_rc_ != RS_OK) return rs_try_rc_;      \
    } while (0)
