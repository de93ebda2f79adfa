"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/dvbe.h declares; host-only calls agree with the oracle;
parameter validation rejects bad problems before any device work."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    dv.lib()
    return dv


def test_exports_every_declared_symbol(dv):
    names = dv.declared_functions()
    assert len(names) >= 40
    for n in names:
        assert hasattr(dv.lib(), n), n
    assert set(names) == set(dv._SIGS), "binding and header disagree"
    assert "sm_103a" in dv.dvbe_version()


def test_velocity_set_and_faces_match_oracle(dv):
    for rt in (W.RT_LATTICE, 0.7):
        a, b = dv.dvbe_d2q9(rt), O.d2q9(rt)
        np.testing.assert_allclose(a[0], b[0], atol=1e-15)
        np.testing.assert_array_equal(a[1], b[1])
        np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_allclose(dv.dvbe_faces_uniform(17, -1, 2), O.faces_uniform(17, -1, 2), atol=1e-15)
    np.testing.assert_allclose(dv.dvbe_faces_tanh(33, 0, 1, 1.5), O.faces_tanh(33, 0, 1, 1.5), atol=1e-15)
    np.testing.assert_allclose(dv.dvbe_faces_geometric(20, 0.0, 1e-3, 1.02),
                               O.faces_geometric(20, 0.0, 1e-3, 1.02), rtol=1e-14)


def test_mesh_geometry_and_cfl(dv):
    xf, yf = W.tanh_faces(12, 0, 1, 1.5), W.geometric_faces(9, 0, 0.01, 1.1)
    m = dv.dvbe_mesh_create(xf, yf)
    try:
        xc, yc, vol = dv.dvbe_mesh_geometry(m, 12, 9)
        np.testing.assert_allclose(xc, W.centres(xf), atol=1e-16)
        np.testing.assert_allclose(vol, np.outer(np.diff(yf), np.diff(xf)), rtol=1e-15)
        dt = dv.dvbe_dt_from_cfl(m, W.RT_LATTICE, 0.5)
        assert dt == pytest.approx(O.dt_from_cfl(xf, yf, W.RT_LATTICE, 0.5), rel=1e-15)
    finally:
        dv.dvbe_mesh_destroy(m)


def test_bad_meshes_rejected(dv):
    with pytest.raises(dv.DvbeError) as e:
        dv.dvbe_mesh_create([0, 1, 0.5], [0, 1, 2])
    assert e.value.status == dv.DVBE_ERR_INVALID_ARG
    with pytest.raises(dv.DvbeError):
        dv.dvbe_mesh_create([0, 1], [0, 1, 2])  # nx = 1


def _create_status(dv, case, **kw):
    try:
        s = dv.Solver(case, **kw)
    except dv.DvbeError as e:
        return e.status
    s.close()
    return dv.DVBE_OK


def test_validation_before_device_work(dv):
    """These are refused by host checks, so they run without a GPU."""
    case, _ = W.taylor_green_box(16)
    bad = dict(case, dt=case["dt"] * 2.5)  # CFL 1.25 (Eq. eq:cfl)
    assert _create_status(dv, bad) == dv.DVBE_ERR_CFL
    assert _create_status(dv, dict(case, tau=-1.0)) == dv.DVBE_ERR_INVALID_ARG
    half = dict(case, bc=[case["bc"][0], [W.wall()], case["bc"][2], case["bc"][3]])
    assert _create_status(dv, half) == dv.DVBE_ERR_INVALID_ARG  # periodic W without E
    gap = dict(case, bc=[[W.wall()], [W.wall()], [("wall", 0.0, 1.0, 1, 0, 0)], [W.wall()]])
    assert _create_status(dv, gap) == dv.DVBE_ERR_INVALID_ARG  # S side not covered
    cav, _ = W.cavity(16)
    assert _create_status(dv, dict(cav, scheme="bkg"), bkg_fd=True) == dv.DVBE_ERR_UNSUPPORTED
    # the finite-difference form is BKG only, not the collision-free faces
    assert _create_status(dv, dict(case, scheme="cfree_upwind"), bkg_fd=True) == dv.DVBE_ERR_UNSUPPORTED
    # scheme codes beyond the four of dvbe_scheme
    assert _create_status(dv, dict(case, scheme=4)) == dv.DVBE_ERR_INVALID_ARG
    assert _create_status(dv, dict(case, scheme=-1)) == dv.DVBE_ERR_INVALID_ARG
    assert "CFL" in (lambda: (_create_status(dv, bad), dv.dvbe_last_error())[1])()


def test_quad_mesh_cells_and_cfl_match_oracle(dv):
    """dvbe_mesh_create_quad / dvbe_mesh_cells / dvbe_dt_from_cfl on
    distorted meshes against the oracle's own quad geometry."""
    for X, Y in (W.quad_random_interior(9, 7, 2, amp=0.3), W.quad_wavy_periodic(12, amp=0.05)):
        ny, nx = X.shape[0] - 1, X.shape[1] - 1
        m = dv.dvbe_mesh_create_quad(X, Y)
        try:
            xc, yc, vol = dv.dvbe_mesh_cells(m, nx, ny)
            case = dict(nx=nx, ny=ny, X=X, Y=Y, RT=W.RT_LATTICE, tau=0.1, dt=0.01, bc=W.periodic_bc())
            oxc, oyc, ovol = O.quad_geometry(case)
            np.testing.assert_allclose(xc, oxc, rtol=0, atol=1e-15)
            np.testing.assert_allclose(yc, oyc, rtol=0, atol=1e-15)
            np.testing.assert_allclose(vol, ovol, rtol=1e-14)
            assert abs(dv.dvbe_dt_from_cfl(m, W.RT_LATTICE, 0.5) / O.quad_dt_from_cfl(case, 0.5) - 1) < 1e-15
            with pytest.raises(dv.DvbeError) as e:
                dv.dvbe_mesh_geometry(m, nx, ny)
            assert e.value.status == dv.DVBE_ERR_UNSUPPORTED
        finally:
            dv.dvbe_mesh_destroy(m)
    # tensor meshes answer dvbe_mesh_cells too
    xf, yf = W.tanh_faces(6, 0, 1, 1.2), W.uniform_faces(5, 0, 2)
    m = dv.dvbe_mesh_create(xf, yf)
    xc, yc, vol = dv.dvbe_mesh_cells(m, 6, 5)
    dv.dvbe_mesh_destroy(m)
    np.testing.assert_allclose(xc[0], W.centres(xf), atol=1e-15)
    np.testing.assert_allclose(yc[:, 0], W.centres(yf), atol=1e-15)
    np.testing.assert_allclose(vol, np.outer(np.diff(yf), np.diff(xf)), rtol=1e-15)


def test_bad_quad_meshes_rejected(dv):
    X, Y = W.quad_random_interior(6, 5, 1, amp=0.2)
    for Xb, Yb in ((X[:, ::-1], Y[:, ::-1]),              # clockwise cells
                   (np.where(np.isin(np.arange(X.size).reshape(X.shape), [9]), np.nan, X), Y)):
        with pytest.raises(dv.DvbeError) as e:
            dv.dvbe_mesh_create_quad(np.ascontiguousarray(Xb), np.ascontiguousarray(Yb))
        assert e.value.status == dv.DVBE_ERR_INVALID_ARG
    with pytest.raises(dv.DvbeError):
        dv.dvbe_mesh_create_quad(X[:2, :1], Y[:2, :1])    # fewer than 2 cells a side
