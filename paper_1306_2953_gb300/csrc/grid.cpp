// Host part of the library: grids (Sec. II), point ordering by small
// parallelepipeds (Sec. V.A) and Kleinman-Bylander projector tables
// (Sec. V.C, Eq. 4).  Integer decisions (which lattice points belong to the
// grid or to a projector sphere) use plain IEEE double arithmetic in a fixed
// order; this file is compiled without floating-point contraction.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <limits>
#include <new>

#include "common.h"

namespace rs {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

const std::string &last_error() { return g_err; }

// Margin of the point map: the star stencil's half-width.
static const int MARGIN = 4;
// Tile of the tile-column order: 16 points along map axis 2, 8 along axis 1.
static const int TILE_X = 16, TILE_Y = 8;

static bool valid_order(int order) {
    return order == 0 || order == 1 || order == 2 || order == 4 || order == 8 || order == RS_ORDER_MORTON ||
           order == RS_ORDER_TILECOL;
}

// Interleaves the bits of (u, v, w), u the most significant at every level.
static uint64_t morton_key(uint64_t u, uint64_t v, uint64_t w) {
    uint64_t k = 0;
    for (int b = 20; b >= 0; --b) k = (k << 3) | (((u >> b) & 1) << 2) | (((v >> b) & 1) << 1) | ((w >> b) & 1);
    return k;
}

// Orders the marked lattice points and fills ijk / map.  mask covers the
// lattice box [lo, lo+ext) (ext[2] fastest).  Orders (map coordinates u, v, w
// along axes 0, 1, 2): bricks of order^3 points in brick raster order, each
// brick lexicographic (order 1: plain lexicographic); the Morton Z-curve; or
// tile columns of TILE_X x TILE_Y points along axes 2 and 1 in raster
// order, each column plane by plane along axis 0, each plane row by row.
static int finish_grid(rs_grid *g, const std::vector<uint8_t> &mask, const int64_t lo[3], const int64_t ext[3],
                       int order) {
    int64_t mn[3] = {std::numeric_limits<int64_t>::max(), std::numeric_limits<int64_t>::max(),
                     std::numeric_limits<int64_t>::max()};
    int64_t mx[3] = {std::numeric_limits<int64_t>::min(), std::numeric_limits<int64_t>::min(),
                     std::numeric_limits<int64_t>::min()};
    int64_t count = 0;
    for (int64_t a = 0; a < ext[0]; ++a)
        for (int64_t b = 0; b < ext[1]; ++b)
            for (int64_t c = 0; c < ext[2]; ++c)
                if (mask[(a * ext[1] + b) * ext[2] + c]) {
                    ++count;
                    int64_t p[3] = {lo[0] + a, lo[1] + b, lo[2] + c};
                    for (int d = 0; d < 3; ++d) {
                        mn[d] = std::min(mn[d], p[d]);
                        mx[d] = std::max(mx[d], p[d]);
                    }
                }
    if (count == 0) return fail(RS_EINVAL, "grid has no points");
    if (count > (int64_t)std::numeric_limits<int32_t>::max()) return fail(RS_EINVAL, "grid too large");
    int64_t dims[3], msize = 1;
    for (int d = 0; d < 3; ++d) {
        g->origin[d] = (int32_t)(mn[d] - MARGIN);
        dims[d] = mx[d] - mn[d] + 1 + 2 * MARGIN;
        g->dims[d] = (int32_t)dims[d];
        msize *= dims[d];
    }
    if (msize > (int64_t)std::numeric_limits<int32_t>::max()) return fail(RS_EINVAL, "point map too large");
    try {
        g->map.assign((size_t)msize, -1);
        g->ijk.resize((size_t)count * 3);
    } catch (const std::bad_alloc &) {
        return fail(RS_ENOMEM, "host allocation failed");
    }
    g->npts = count;
    g->order = order == 0 ? 4 : order;
    int64_t next = 0;
    // numbers map position (u, v, w) if it is a marked lattice point
    auto take = [&](int64_t u, int64_t v, int64_t w) {
        const int64_t p[3] = {g->origin[0] + u, g->origin[1] + v, g->origin[2] + w};
        const int64_t a = p[0] - lo[0], b = p[1] - lo[1], c = p[2] - lo[2];
        if (a < 0 || b < 0 || c < 0 || a >= ext[0] || b >= ext[1] || c >= ext[2]) return;
        if (!mask[(a * ext[1] + b) * ext[2] + c]) return;
        g->map[(size_t)((u * dims[1] + v) * dims[2] + w)] = (int32_t)next;
        g->ijk[3 * next + 0] = (int32_t)p[0];
        g->ijk[3 * next + 1] = (int32_t)p[1];
        g->ijk[3 * next + 2] = (int32_t)p[2];
        ++next;
    };
    if (g->order > 0) {
        const int B = g->order;
        int64_t nb[3];
        for (int d = 0; d < 3; ++d) nb[d] = (dims[d] + B - 1) / B;
        for (int64_t B0 = 0; B0 < nb[0]; ++B0)
            for (int64_t B1 = 0; B1 < nb[1]; ++B1)
                for (int64_t B2 = 0; B2 < nb[2]; ++B2)
                    for (int64_t u = B0 * B; u < std::min(dims[0], (B0 + 1) * B); ++u)
                        for (int64_t v = B1 * B; v < std::min(dims[1], (B1 + 1) * B); ++v)
                            for (int64_t w = B2 * B; w < std::min(dims[2], (B2 + 1) * B); ++w) take(u, v, w);
    } else if (g->order == RS_ORDER_TILECOL) {
        for (int64_t t1 = 0; t1 < (dims[1] + TILE_Y - 1) / TILE_Y; ++t1)
            for (int64_t t2 = 0; t2 < (dims[2] + TILE_X - 1) / TILE_X; ++t2)
                for (int64_t u = 0; u < dims[0]; ++u)
                    for (int64_t v = t1 * TILE_Y; v < std::min(dims[1], (t1 + 1) * TILE_Y); ++v)
                        for (int64_t w = t2 * TILE_X; w < std::min(dims[2], (t2 + 1) * TILE_X); ++w) take(u, v, w);
    } else {   // Morton
        std::vector<std::pair<uint64_t, int64_t>> keys;
        try {
            keys.reserve((size_t)count);
        } catch (const std::bad_alloc &) {
            return fail(RS_ENOMEM, "host allocation failed");
        }
        for (int64_t u = 0; u < dims[0]; ++u)
            for (int64_t v = 0; v < dims[1]; ++v)
                for (int64_t w = 0; w < dims[2]; ++w) {
                    const int64_t a = g->origin[0] + u - lo[0], b = g->origin[1] + v - lo[1], c = g->origin[2] + w - lo[2];
                    if (a < 0 || b < 0 || c < 0 || a >= ext[0] || b >= ext[1] || c >= ext[2]) continue;
                    if (mask[(a * ext[1] + b) * ext[2] + c]) keys.emplace_back(morton_key(u, v, w), (u * dims[1] + v) * dims[2] + w);
                }
        std::sort(keys.begin(), keys.end());
        for (const auto &k : keys) {
            const int64_t m = k.second, w = m % dims[2], v = (m / dims[2]) % dims[1], u = m / (dims[2] * dims[1]);
            take(u, v, w);
        }
    }
    return next == count ? RS_OK : fail(RS_EINVAL, "grid ordering lost points");
}

}  // namespace rs

using rs::fail;

extern "C" int rs_last_error(char *buf, size_t len) {
    const std::string &e = rs::last_error();
    if (buf && len) {
        size_t n = std::min(len - 1, e.size());
        memcpy(buf, e.data(), n);
        buf[n] = 0;
    }
    return (int)e.size();
}

extern "C" const char *rs_version(void) { return "rsdft 0.1 sm_103a"; }

extern "C" int rs_grid_create_spheres(const double *xyz, int n_atoms, double radius, double h, int order,
                                      rs_grid **out) {
    if (!xyz || !out || n_atoms < 1) return fail(RS_EINVAL, "rs_grid_create_spheres: bad arguments");
    if (!rs::valid_order(order)) return fail(RS_EINVAL, "rs_grid_create_spheres: bad point order %d", order);
    if (!(radius > 0) || !(h > 0) || !std::isfinite(radius) || !std::isfinite(h))
        return fail(RS_EINVAL, "rs_grid_create_spheres: radius and h must be positive");
    for (int i = 0; i < 3 * n_atoms; ++i)
        if (!std::isfinite(xyz[i])) return fail(RS_EINVAL, "rs_grid_create_spheres: non-finite coordinate");
    *out = nullptr;
    double amin[3], amax[3];
    for (int d = 0; d < 3; ++d) {
        amin[d] = amax[d] = xyz[d];
        for (int a = 1; a < n_atoms; ++a) {
            amin[d] = std::min(amin[d], xyz[3 * a + d]);
            amax[d] = std::max(amax[d], xyz[3 * a + d]);
        }
    }
    int64_t lo[3], ext[3], total = 1;
    for (int d = 0; d < 3; ++d) {
        double l = std::floor((amin[d] - radius) / h) - 1, u = std::ceil((amax[d] + radius) / h) + 1;
        if (u - l > 1e6) return fail(RS_EINVAL, "rs_grid_create_spheres: grid too large");
        lo[d] = (int64_t)l;
        ext[d] = (int64_t)u - lo[d] + 1;
        total *= ext[d];
    }
    if (total > (int64_t)1 << 33) return fail(RS_EINVAL, "rs_grid_create_spheres: grid too large");
    std::vector<uint8_t> mask;
    try {
        mask.assign((size_t)total, 0);
    } catch (const std::bad_alloc &) {
        return fail(RS_ENOMEM, "host allocation failed");
    }
    const double r2 = radius * radius;
    for (int A = 0; A < n_atoms; ++A) {
        const double X = xyz[3 * A], Y = xyz[3 * A + 1], Z = xyz[3 * A + 2];
        int64_t a0 = std::max<int64_t>(lo[0], (int64_t)std::floor((X - radius) / h) - 1);
        int64_t a1 = std::min<int64_t>(lo[0] + ext[0] - 1, (int64_t)std::ceil((X + radius) / h) + 1);
        int64_t b0 = std::max<int64_t>(lo[1], (int64_t)std::floor((Y - radius) / h) - 1);
        int64_t b1 = std::min<int64_t>(lo[1] + ext[1] - 1, (int64_t)std::ceil((Y + radius) / h) + 1);
        int64_t c0 = std::max<int64_t>(lo[2], (int64_t)std::floor((Z - radius) / h) - 1);
        int64_t c1 = std::min<int64_t>(lo[2] + ext[2] - 1, (int64_t)std::ceil((Z + radius) / h) + 1);
        for (int64_t i = a0; i <= a1; ++i) {
            const double dx = h * (double)i - X;
            for (int64_t j = b0; j <= b1; ++j) {
                const double dy = h * (double)j - Y;
                for (int64_t k = c0; k <= c1; ++k) {
                    const double dz = h * (double)k - Z;
                    const double d2 = (dx * dx + dy * dy) + dz * dz;
                    if (d2 <= r2) mask[(size_t)(((i - lo[0]) * ext[1] + (j - lo[1])) * ext[2] + (k - lo[2]))] = 1;
                }
            }
        }
    }
    rs_grid *g = new (std::nothrow) rs_grid;
    if (!g) return fail(RS_ENOMEM, "host allocation failed");
    g->h = h;
    int rc = rs::finish_grid(g, mask, lo, ext, order);
    if (rc != RS_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return RS_OK;
}

extern "C" int rs_grid_create_box(int n0, int n1, int n2, double h, int order, rs_grid **out) {
    if (!out || n0 < 1 || n1 < 1 || n2 < 1 || !(h > 0) || !std::isfinite(h))
        return fail(RS_EINVAL, "rs_grid_create_box: bad arguments");
    if (!rs::valid_order(order)) return fail(RS_EINVAL, "rs_grid_create_box: bad point order %d", order);
    if ((int64_t)n0 * n1 * n2 > (int64_t)1 << 30) return fail(RS_EINVAL, "rs_grid_create_box: grid too large");
    *out = nullptr;
    int64_t lo[3] = {0, 0, 0}, ext[3] = {n0, n1, n2};
    std::vector<uint8_t> mask((size_t)n0 * n1 * n2, 1);
    rs_grid *g = new (std::nothrow) rs_grid;
    if (!g) return fail(RS_ENOMEM, "host allocation failed");
    g->h = h;
    g->center[0] = (n0 - 1) / 2.0;
    g->center[1] = (n1 - 1) / 2.0;
    g->center[2] = (n2 - 1) / 2.0;
    int rc = rs::finish_grid(g, mask, lo, ext, order);
    if (rc != RS_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return RS_OK;
}

extern "C" int rs_grid_info(const rs_grid *g, int64_t *npts, int32_t origin[3], int32_t dims[3], double *h) {
    if (!g) return fail(RS_EINVAL, "rs_grid_info: null grid");
    if (npts) *npts = g->npts;
    if (origin) memcpy(origin, g->origin, sizeof(g->origin));
    if (dims) memcpy(dims, g->dims, sizeof(g->dims));
    if (h) *h = g->h;
    return RS_OK;
}

extern "C" int rs_grid_ijk(const rs_grid *g, int32_t *ijk_out) {
    if (!g || !ijk_out) return fail(RS_EINVAL, "rs_grid_ijk: null argument");
    memcpy(ijk_out, g->ijk.data(), g->ijk.size() * sizeof(int32_t));
    return RS_OK;
}

extern "C" int rs_grid_coords(const rs_grid *g, double *xyz_out) {
    if (!g || !xyz_out) return fail(RS_EINVAL, "rs_grid_coords: null argument");
    for (int64_t p = 0; p < g->npts; ++p)
        for (int d = 0; d < 3; ++d) xyz_out[3 * p + d] = g->coord(d, g->ijk[3 * p + d]);
    return RS_OK;
}

extern "C" int rs_grid_point_map(const rs_grid *g, int32_t *map_out) {
    if (!g || !map_out) return fail(RS_EINVAL, "rs_grid_point_map: null argument");
    memcpy(map_out, g->map.data(), g->map.size() * sizeof(int32_t));
    return RS_OK;
}

extern "C" int rs_grid_destroy(rs_grid *g) {
    delete g;
    return RS_OK;
}

// ------------------------------------------------------------ projectors --

extern "C" int rs_proj_create(const rs_grid *g, const rs_projector_spec *spec, rs_proj **out) {
    if (!g || !spec || !out || spec->n_atoms < 0 || (spec->n_atoms > 0 && (!spec->xyz || !spec->E)))
        return fail(RS_EINVAL, "rs_proj_create: bad arguments");
    if (!(spec->r_c > 0) || !(spec->r_cut > 0)) return fail(RS_EINVAL, "rs_proj_create: r_c and r_cut must be > 0");
    *out = nullptr;
    rs_proj *pr = new (std::nothrow) rs_proj;
    if (!pr) return fail(RS_ENOMEM, "host allocation failed");
    const int n = spec->n_atoms;
    const double h = g->h, rc2 = spec->r_cut * spec->r_cut, dV = h * h * h;
    const double inv2w = 1.0 / (2.0 * spec->r_c * spec->r_c);
    pr->n_atoms = n;
    pr->off.assign((size_t)n + 1, 0);
    pr->E.resize((size_t)n * 4);
    struct Ent {
        int32_t p;
        double dx, dy, dz, d2;
    };
    std::vector<Ent> ents;
    for (int A = 0; A < n; ++A) {
        const double X = spec->xyz[3 * A], Y = spec->xyz[3 * A + 1], Z = spec->xyz[3 * A + 2];
        const double Es = spec->E[2 * A], Ep = spec->E[2 * A + 1];
        pr->E[4 * A] = Es;
        pr->E[4 * A + 1] = pr->E[4 * A + 2] = pr->E[4 * A + 3] = Ep;
        ents.clear();
        int64_t lo[3], hi[3];
        const double P[3] = {X, Y, Z};
        for (int d = 0; d < 3; ++d) {
            // lattice range covering the sphere: coord(i) = (i - center) h
            lo[d] = (int64_t)std::floor((P[d] - spec->r_cut) / h + g->center[d]) - 1;
            hi[d] = (int64_t)std::ceil((P[d] + spec->r_cut) / h + g->center[d]) + 1;
            lo[d] = std::max<int64_t>(lo[d], g->origin[d]);
            hi[d] = std::min<int64_t>(hi[d], (int64_t)g->origin[d] + g->dims[d] - 1);
        }
        for (int64_t i = lo[0]; i <= hi[0]; ++i) {
            const double dx = g->coord(0, (int32_t)i) - X;
            for (int64_t j = lo[1]; j <= hi[1]; ++j) {
                const double dy = g->coord(1, (int32_t)j) - Y;
                for (int64_t k = lo[2]; k <= hi[2]; ++k) {
                    const int32_t p = g->map[(size_t)(((i - g->origin[0]) * g->dims[1] + (j - g->origin[1])) *
                                                          g->dims[2] + (k - g->origin[2]))];
                    if (p < 0) continue;
                    const double dz = g->coord(2, (int32_t)k) - Z;
                    const double d2 = (dx * dx + dy * dy) + dz * dz;
                    if (d2 <= rc2) ents.push_back({p, dx, dy, dz, d2});
                }
            }
        }
        std::sort(ents.begin(), ents.end(), [](const Ent &a, const Ent &b) { return a.p < b.p; });
        const size_t base = pr->idx.size();
        pr->idx.resize(base + ents.size());
        pr->gam.resize((base + ents.size()) * 4);
        double nrm[4] = {0, 0, 0, 0};
        for (size_t e = 0; e < ents.size(); ++e) {
            const double gv = std::exp(-ents[e].d2 * inv2w);
            double v[4] = {gv, ents[e].dx * gv, ents[e].dy * gv, ents[e].dz * gv};
            pr->idx[base + e] = ents[e].p;
            for (int q = 0; q < 4; ++q) {
                pr->gam[(base + e) * 4 + q] = v[q];
                nrm[q] += v[q] * v[q];
            }
        }
        for (int q = 0; q < 4; ++q) nrm[q] = nrm[q] > 0 ? 1.0 / std::sqrt(dV * nrm[q]) : 0.0;
        for (size_t e = 0; e < ents.size(); ++e)
            for (int q = 0; q < 4; ++q) pr->gam[(base + e) * 4 + q] *= nrm[q];
        pr->off[(size_t)A + 1] = (int64_t)pr->idx.size();
    }
    *out = pr;
    return RS_OK;
}

extern "C" int rs_proj_info(const rs_proj *pr, int32_t *n_atoms, int64_t *n_entries) {
    if (!pr) return fail(RS_EINVAL, "rs_proj_info: null handle");
    if (n_atoms) *n_atoms = pr->n_atoms;
    if (n_entries) *n_entries = (int64_t)pr->idx.size();
    return RS_OK;
}

extern "C" int rs_proj_tables(const rs_proj *pr, int64_t *sph_off, int32_t *sph_idx, double *gamma) {
    if (!pr) return fail(RS_EINVAL, "rs_proj_tables: null handle");
    if (sph_off) memcpy(sph_off, pr->off.data(), pr->off.size() * sizeof(int64_t));
    if (sph_idx) memcpy(sph_idx, pr->idx.data(), pr->idx.size() * sizeof(int32_t));
    if (gamma) memcpy(gamma, pr->gam.data(), pr->gam.size() * sizeof(double));
    return RS_OK;
}

extern "C" int rs_proj_destroy(rs_proj *pr) {
    delete pr;
    return RS_OK;
}
