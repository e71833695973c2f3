"""GPU parity of the measurement operator (Phi = G F Z S, Sec. 1 measurement
equation) against the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, TOL, make_plan, np_cplx, np_real, rel, t_cplx, t_real
from oracle import nufft as onf
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, M, J, R, dtype
    (16, 16, 300, 4, 1, pk.PURIFY_F32),
    (32, 32, 4099, 6, 3, pk.PURIFY_F32),
    (64, 32, 5001, 5, 2, pk.PURIFY_F32),
    (64, 64, 8192, 4, 1, pk.PURIFY_F64),
    (32, 64, 3001, 6, 4, pk.PURIFY_F64),
    (128, 128, 40000, 8, 5, pk.PURIFY_F32),
    (16, 16, 1, 6, 1, pk.PURIFY_F32),
]


def oracle_plan(nx, ny, u, v, J):
    return onf.NufftPlan(nx, ny, u.astype(np.float64), v.astype(np.float64), J)


@pytest.mark.parametrize("nx,ny,M,J,R,dtype", CASES)
def test_phi_matches_oracle(nx, ny, M, J, R, dtype):
    plan, u, v, _ = make_plan(nx, ny, M, J, R=R, dtype=dtype, seed=nx + M)
    x = np.random.default_rng(1).standard_normal((ny, nx)).astype(np_real(dtype))
    y = torch.empty(M, dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi(plan, torch.from_numpy(x).to(DEV), y)
    want = onf.phi(oracle_plan(nx, ny, u, v, J), x.astype(np.float64))
    assert rel(y.cpu().numpy(), want) <= TOL[dtype]


@pytest.mark.parametrize("nx,ny,M,J,R,dtype", CASES)
def test_phi_adj_matches_oracle(nx, ny, M, J, R, dtype):
    plan, u, v, _ = make_plan(nx, ny, M, J, R=R, dtype=dtype, seed=nx + M + 1)
    g = np.random.default_rng(2)
    y = (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np_cplx(dtype))
    x = torch.empty((ny, nx), dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi_adj(plan, torch.from_numpy(y).to(DEV), x)
    want = onf.phi_adj(oracle_plan(nx, ny, u, v, J), y.astype(np.complex128))
    assert rel(x.cpu().numpy(), want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [pk.PURIFY_F32, pk.PURIFY_F64])
@pytest.mark.parametrize("K", [16, 32, 128, 512, 2048])
def test_fft2_matches_oracle(K, dtype):
    n = K // 2
    plan, _, _, _ = make_plan(n, n, 64, 4, dtype=dtype, seed=K)
    g = np.random.default_rng(K)
    X = (g.standard_normal((K, K)) + 1j * g.standard_normal((K, K))).astype(np_cplx(dtype))
    for inv in (False, True):
        t = torch.from_numpy(X).to(DEV)
        pk.purify_fft2(plan, t, inv)
        want = onf.ifft2_unnormalised(X.astype(np.complex128)) if inv else onf.fft2(X.astype(np.complex128))
        assert rel(t.cpu().numpy(), want) <= 3 * TOL[dtype]


def test_adjoint_identity_on_gpu():
    # <Phi x, y> = <x, Re Phi^H y> for real x, computed from GPU outputs only
    nx = ny = 64
    M = 20000
    plan, _, _, _ = make_plan(nx, ny, M, 6, R=2, seed=11)
    g = np.random.default_rng(3)
    x = torch.from_numpy(g.standard_normal((ny, nx)).astype(np.float32)).to(DEV)
    yv = torch.from_numpy((g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex64)).to(DEV)
    Ax = torch.empty(M, dtype=torch.complex64, device=DEV)
    Ay = torch.empty((ny, nx), dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, x, Ax)
    pk.purify_phi_adj(plan, yv, Ay)
    lhs = torch.vdot(yv.to(torch.complex128), Ax.to(torch.complex128)).real.item()
    rhs = torch.sum(x.double() * Ay.real.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_band_edges_and_tiny_tiles():
    # coordinates at -pi and just below +pi wrap around the grid
    nx = ny = 32
    u = np.array([-np.pi, np.nextafter(np.float32(np.pi), 0), 0.0, -np.pi, 1.0], dtype=np.float32)
    v = np.array([0.3, -np.pi, np.nextafter(np.float32(np.pi), 0), -np.pi, -1.0], dtype=np.float32)
    for tile in (8, 16, 64):
        plan = pk.Plan(nx, ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=6, levels=2,
                       tile=tile)
        x = np.random.default_rng(4).standard_normal((ny, nx)).astype(np.float32)
        y = torch.empty(u.size, dtype=torch.complex64, device=DEV)
        pk.purify_phi(plan, torch.from_numpy(x).to(DEV), y)
        op = oracle_plan(nx, ny, u, v, 6)
        assert rel(y.cpu().numpy(), onf.phi(op, x.astype(np.float64))) <= 1e-5
        g = np.random.default_rng(tile)
        yv = (g.standard_normal(u.size) + 1j * g.standard_normal(u.size)).astype(np.complex64)
        xa = torch.empty((ny, nx), dtype=torch.complex64, device=DEV)
        pk.purify_phi_adj(plan, torch.from_numpy(yv).to(DEV), xa)
        assert rel(xa.cpu().numpy(), onf.phi_adj(op, yv.astype(np.complex128))) <= 1e-5


def test_dense_bin_uses_many_subproblems():
    # every visibility in one grid tile: the tile is split into many
    # subproblems that add into the same cells
    nx = ny = 64
    M = 30000
    g = np.random.default_rng(5)
    u = g.uniform(-0.05, 0.05, M).astype(np.float32)
    v = g.uniform(-0.05, 0.05, M).astype(np.float32)
    plan = pk.Plan(nx, ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=6, levels=2)
    yv = (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex64)
    xa = torch.empty((ny, nx), dtype=torch.complex64, device=DEV)
    pk.purify_phi_adj(plan, torch.from_numpy(yv).to(DEV), xa)
    want = onf.phi_adj(oracle_plan(nx, ny, u, v, 6), yv.astype(np.complex128))
    assert rel(xa.cpu().numpy(), want) <= 1e-5


def test_host_pointers_match_device_pointers():
    nx = ny = 32
    M = 1000
    plan, u, v, _ = make_plan(nx, ny, M, 6, seed=6)
    x = np.random.default_rng(7).standard_normal((ny, nx)).astype(np.float32)
    y_host = np.empty(M, dtype=np.complex64)
    pk.purify_phi(plan, x, y_host)
    y_dev = torch.empty(M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, torch.from_numpy(x).to(DEV), y_dev)
    assert np.array_equal(y_host, y_dev.cpu().numpy())


def test_full_size_sampled_outputs():
    # the 256 x 256, M = 655360, J = 6, 8-block workload; sampled visibilities
    # are checked one by one against the oracle on the same (u, v)
    wl = synth.WORKLOADS["sara256_r8"]
    x, u, v, offs, _ = wl.draw()
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs)
    xf = x.astype(np.float32)
    y = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, torch.from_numpy(xf).to(DEV), y)
    idx = np.random.default_rng(8).choice(wl.M, 3000, replace=False)
    op = oracle_plan(wl.nx, wl.ny, u[idx], v[idx], wl.J)
    want = onf.phi(op, xf.astype(np.float64))
    assert rel(y.cpu().numpy()[idx], want) <= 1e-5
    # adjoint identity at full size
    g = np.random.default_rng(9)
    yv = torch.from_numpy((g.standard_normal(wl.M) + 1j * g.standard_normal(wl.M)).astype(np.complex64)).to(DEV)
    xa = torch.empty((wl.ny, wl.nx), dtype=torch.complex64, device=DEV)
    pk.purify_phi_adj(plan, yv, xa)
    lhs = torch.vdot(yv.to(torch.complex128), y.to(torch.complex128)).real.item()
    rhs = torch.sum(torch.from_numpy(xf).to(DEV).double() * xa.real.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("grid_mode", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("nx,M,J,R,dtype,tile", [
    (64, 30011, 6, 3, pk.PURIFY_F32, 0),
    (64, 30011, 6, 3, pk.PURIFY_F32, 16),
    (128, 70001, 4, 2, pk.PURIFY_F32, 64),
    (32, 4099, 7, 2, pk.PURIFY_F64, 0),
    (16, 5, 5, 1, pk.PURIFY_F32, 0),
])
def test_phi_adj_both_decompositions(nx, M, J, R, dtype, tile, grid_mode):
    # G^H by tile subproblems, by first-tap-cell runs and by lanes (3: a run
    # per lane, 4: per lane pair, 5: per lane pair, runs grouped by tile, 6:
    # per lane pair with stored patches summed in a fixed order), each against the
    # oracle in caller order: several tiles, runs cut at their length cap, a
    # ragged last run set, an odd J and a handful of visibilities; also G
    # (Phi) and the normal operator of each decomposition
    if grid_mode >= 3 and (dtype != pk.PURIFY_F32 or J > 6):
        pytest.skip("lanes are FP32 with J <= 6 only")
    plan, u, v, _ = make_plan(nx, nx, M, J, R=R, dtype=dtype, seed=nx + M + grid_mode, tile=tile,
                              grid_mode=grid_mode)
    assert plan.info.grid_mode == grid_mode
    g = np.random.default_rng(M)
    y = (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np_cplx(dtype))
    x = torch.empty((nx, nx), dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi_adj(plan, torch.from_numpy(y).to(DEV), x)
    op = oracle_plan(nx, nx, u, v, J)
    want = onf.phi_adj(op, y.astype(np.complex128))
    assert rel(x.cpu().numpy(), want) <= TOL[dtype]
    xr = np.random.default_rng(M + 1).standard_normal((nx, nx)).astype(np_real(dtype))
    yg = torch.empty(M, dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi(plan, torch.from_numpy(xr).to(DEV), yg)
    assert rel(yg.cpu().numpy(), onf.phi(op, xr.astype(np.float64))) <= TOL[dtype]
    out = torch.empty((nx, nx), dtype=t_real(dtype), device=DEV)
    pk.purify_phi_normal(plan, torch.from_numpy(xr).to(DEV), out)
    want_n = np.real(onf.phi_adj(op, onf.phi(op, xr.astype(np.float64))))
    assert rel(out.cpu().numpy(), want_n) <= TOL[dtype]


@pytest.mark.parametrize("grid_mode", [1, 2, 3, 4, 5, 6])
def test_phi_adj_single_cell_runs(grid_mode):
    # every visibility in a handful of cells: runs longer than the cap are
    # cut and flushed into the same cells
    nx = 32
    M = 20000
    g = np.random.default_rng(12)
    u = (np.round(g.uniform(-3, 3, M)) * (2 * np.pi / 64) + 1e-4).astype(np.float32)
    v = (np.round(g.uniform(-3, 3, M)) * (2 * np.pi / 64) - 1e-4).astype(np.float32)
    plan = pk.Plan(nx, nx, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=6, levels=2,
                   grid_mode=grid_mode)
    yv = (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex64)
    xa = torch.empty((nx, nx), dtype=torch.complex64, device=DEV)
    pk.purify_phi_adj(plan, torch.from_numpy(yv).to(DEV), xa)
    want = onf.phi_adj(oracle_plan(nx, nx, u, v, 6), yv.astype(np.complex128))
    assert rel(xa.cpu().numpy(), want) <= 1e-5
