"""Host-side library logic against the oracle (no GPU needed): the grid's
point set and map (bit-exact), the brick ordering, the projector sphere
lists (bit-exact) and their coefficients, and argument checking."""
import numpy as np
import pytest

import workloads as wl
from oracle import grid as og, hamiltonian as oh
from paper_1306_2953_gb300 import api
from paper_1306_2953_gb300._lib import RS_EINVAL, RS_ORDER_MORTON, RS_ORDER_TILECOL, RsError
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS, lib_to_oracle_index


def _same_points(lg, og_):
    lib_ijk = lg.ijk()
    assert lg.npts == og_.npts
    assert set(map(tuple, lib_ijk.tolist())) == set(map(tuple, og_.ijk.tolist()))
    return lib_ijk


@pytest.mark.parametrize("spec", [wl.MOL20.system, wl.MoleculeSpec(7, 5.0, 1.5, 2.5, 0.41, 11)])
def test_sphere_grid_bit_exact(spec):
    atoms = wl.atom_positions(spec)
    lg = api.Grid.spheres(atoms, spec.radius, spec.h)
    ref = og.sphere_union_grid(atoms, spec.radius, spec.h)
    lib_ijk = _same_points(lg, ref)
    # the point map is consistent with the coordinates and -1 elsewhere
    npts, origin, dims, h = lg.info()
    mp = lg.point_map()
    assert mp.shape == tuple(dims)
    rel = lib_ijk - np.array(origin)
    assert np.array_equal(mp[rel[:, 0], rel[:, 1], rel[:, 2]], np.arange(npts))
    assert np.sum(mp >= 0) == npts
    # a 4-point margin around every grid point stays inside the map
    assert rel.min() >= 4 and np.all(rel.max(axis=0) <= np.array(dims) - 5)
    # coordinates are h * ijk, bitwise
    assert np.array_equal(lg.coords(), h * lib_ijk.astype(np.float64))


def test_brick_order():
    lg = api.Grid.spheres(np.array([[0.0, 0.0, 0.0]]), 2.0, 0.3)
    _, origin, _, _ = lg.info()
    rel = lg.ijk() - np.array(origin)
    brick = rel // 4
    key = (brick[:, 0] * 10000 + brick[:, 1]) * 10000 + brick[:, 2]
    assert np.all(np.diff(key) >= 0), "points are not grouped brick by brick in brick order"


def _order_key(rel, order, dims):
    """The sort key each point order defines on map coordinates (u, v, w)."""
    u, v, w = (rel[:, d].astype(np.int64) for d in range(3))
    if order > 0:
        b = order
        return ((((u // b) * 10000 + v // b) * 10000 + w // b) * 10000 + (u % b)) * 10000 * 10000 \
            + (v % b) * 10000 + (w % b)
    if order == RS_ORDER_TILECOL:
        nt2 = (dims[2] + 15) // 16
        col = (v // 8) * nt2 + w // 16
        return ((col * 10000 + u) * 100 + v % 8) * 100 + w % 16
    key = np.zeros(len(u), dtype=np.int64)       # Morton: bits interleaved, u most significant
    for bit in range(20, -1, -1):
        key = (key << 3) | (((u >> bit) & 1) << 2) | (((v >> bit) & 1) << 1) | ((w >> bit) & 1)
    return key


@pytest.mark.parametrize("order", [1, 2, 4, 8, RS_ORDER_MORTON, RS_ORDER_TILECOL])
def test_point_orders(order):
    """Every point order numbers the same lattice points (bit-exact against
    the oracle's grid) with a consistent map, in the sequence its definition
    gives: the order's key strictly increases with the point index."""
    spec = wl.MoleculeSpec(7, 5.0, 1.5, 2.5, 0.41, 11)
    atoms = wl.atom_positions(spec)
    lg = api.Grid.spheres(atoms, spec.radius, spec.h, order=order)
    ref = og.sphere_union_grid(atoms, spec.radius, spec.h)
    lib_ijk = _same_points(lg, ref)
    npts, origin, dims, h = lg.info()
    rel = lib_ijk - np.array(origin)
    mp = lg.point_map()
    assert np.array_equal(mp[rel[:, 0], rel[:, 1], rel[:, 2]], np.arange(npts))
    assert np.all(np.diff(_order_key(rel, order, dims)) > 0)
    box = api.Grid.box(9, 6, 20, 0.3, order=order)
    _, bo, bd, _ = box.info()
    brel = box.ijk() - np.array(bo)
    assert box.npts == 9 * 6 * 20 and np.all(np.diff(_order_key(brel, order, bd)) > 0)


def test_point_order_rejects_unknown():
    with pytest.raises(RsError) as e:
        api.Grid.spheres(np.array([[0.0, 0.0, 0.0]]), 2.0, 0.3, order=3)
    assert e.value.code == RS_EINVAL


def test_box_grid_bit_exact():
    lg = api.Grid.box(6, 5, 7, 0.3)
    assert lg.npts == 210
    c = lg.coords()
    ijk = lg.ijk()
    assert np.array_equal(c[:, 1], (ijk[:, 1].astype(np.float64) - 2.0) * 0.3)
    ref = og.box_grid(6, 0.3)
    lg6 = api.Grid.box(6, 6, 6, 0.3)
    idx = lib_to_oracle_index(ref, lg6.ijk())
    assert np.array_equal(lg6.coords(), ref.coords[idx])


def test_projector_tables_match_oracle():
    atoms = np.array(SMALL_ATOMS)
    E = np.array(SMALL_E)
    lg = api.Grid.spheres(atoms, SMALL_RADIUS, SMALL_H)
    ref = og.sphere_union_grid(atoms, SMALL_RADIUS, SMALL_H)
    pr_ref = oh.make_projectors(ref, atoms, E, 1.0, 3.0)
    pr = api.Projectors(lg, atoms, E, 1.0, 3.0)
    off, idx, gam = pr.tables()
    lib_ijk = lg.ijk()
    to_ora = lib_to_oracle_index(ref, lib_ijk)
    for A in range(len(atoms)):
        lib_pts = to_ora[idx[off[A]:off[A + 1]]]
        ora_pts = pr_ref.points(A)
        assert set(lib_pts.tolist()) == set(ora_pts.tolist())      # exact sphere membership
        assert np.all(np.diff(idx[off[A]:off[A + 1]]) > 0)          # ascending library ids
        order = np.argsort(lib_pts)
        g_lib = gam[off[A]:off[A + 1]][order]
        g_ora = pr_ref.gamma(A).T[np.argsort(ora_pts)]
        assert np.abs(g_lib - g_ora).max() < 1e-13 * np.abs(g_ora).max()


def test_argument_errors():
    with pytest.raises(RsError) as e:
        api.Grid.spheres(np.zeros((1, 3)), -1.0, 0.3)
    assert e.value.code == RS_EINVAL
    with pytest.raises(RsError):
        api.Grid.box(0, 4, 4, 0.3)
    with pytest.raises(RsError):
        api.Grid.spheres(np.array([[np.nan, 0.0, 0.0]]), 1.0, 0.3)


def test_library_exports_every_declared_symbol():
    """Every function include/rsdft.h declares is exported by librsdft.so
    (looked up only, never called) and bound by the Python layer."""
    import ctypes
    import os
    import re
    from paper_1306_2953_gb300 import _lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "rsdft.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text)))
    assert len(names) >= 40
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    unbound = [n for n in names if n not in _lib.exported_names()]
    assert not unbound, unbound


# point counts of the seeded molecules (union of 5 Bohr spheres), written
# by the oracle's grid builder; the benchmark's throughput figures refer to
# these sizes
FULL_SIZE_NPTS = {wl.MOL20.name: 103331, wl.MOL100.name: 654520, wl.MOL300.name: 1821562}


@pytest.mark.parametrize("w", [wl.MOL20, wl.MOL100, wl.MOL300], ids=lambda w: w.name)
def test_full_size_grids_bit_exact(w):
    spec = w.system
    atoms = wl.atom_positions(spec)
    lg = api.Grid.spheres(atoms, spec.radius, spec.h)
    ref = og.sphere_union_grid(atoms, spec.radius, spec.h)
    assert lg.npts == ref.npts == FULL_SIZE_NPTS[w.name]
    ijk = lg.ijk()
    assert np.array_equal(ijk[np.lexsort((ijk[:, 2], ijk[:, 1], ijk[:, 0]))], ref.ijk)
    mp = lg.point_map()
    _, origin, _, _ = lg.info()
    rel = ijk - np.array(origin)
    assert np.array_equal(mp[rel[:, 0], rel[:, 1], rel[:, 2]], np.arange(lg.npts))
    assert np.sum(mp >= 0) == lg.npts


def test_full_size_projector_lists_mol100():
    # the 100-atom molecule at full size: every projector sphere list is the
    # oracle's point set, coefficients to FP64 rounding
    spec = wl.MOL100.system
    atoms = wl.atom_positions(spec)
    E = wl.kb_couplings(spec)
    lg = api.Grid.spheres(atoms, spec.radius, spec.h)
    ref = og.sphere_union_grid(atoms, spec.radius, spec.h)
    pr_ref = oh.make_projectors(ref, atoms, E, spec.r_c, spec.r_cut)
    off, idx, gam = api.Projectors(lg, atoms, E, spec.r_c, spec.r_cut).tables()
    assert off[-1] == pr_ref.sph_off[-1]
    to_ora = lib_to_oracle_index(ref, lg.ijk())
    for A in range(spec.n_atoms):
        lib_pts = to_ora[idx[off[A]:off[A + 1]]]
        order = np.argsort(lib_pts)
        assert np.array_equal(lib_pts[order], pr_ref.points(A))
        g_ora = pr_ref.gamma(A).T
        assert np.abs(gam[off[A]:off[A + 1]][order] - g_ora).max() < 1e-13 * np.abs(g_ora).max()


def test_empty_and_invalid_grids_are_rejected():
    # a sphere too small to hold a lattice point, zero or negative sizes,
    # and non-finite positions are all RS_EINVAL (no handle is returned)
    with pytest.raises(RsError) as e:
        api.Grid.spheres(np.array([[0.15, 0.15, 0.15]]), 0.01, 0.3)
    assert e.value.code == RS_EINVAL
    for args in ((np.array([[0.0, 0.0, 0.0]]), -1.0, 0.3), (np.array([[0.0, 0.0, 0.0]]), 2.0, 0.0),
                 (np.array([[np.nan, 0.0, 0.0]]), 2.0, 0.3)):
        with pytest.raises(RsError) as e:
            api.Grid.spheres(*args)
        assert e.value.code == RS_EINVAL
    with pytest.raises(RsError) as e:
        api.Grid.box(0, 4, 4, 0.3)
    assert e.value.code == RS_EINVAL


def test_bounds_checked_build_compiles():
    # the debugging build of the library (index tests in the FP32 H psi
    # kernel) builds beside the normal one and exports the same symbols
    import ctypes
    from paper_1306_2953_gb300 import _lib, build
    path = build.build(bounds_check=True)
    L = ctypes.CDLL(path)
    for name in _lib.exported_names():
        assert hasattr(L, name), name
