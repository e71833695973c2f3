"""The Python binding refuses buffers too small for a plan's call before it
reaches the C ABI (which takes raw pointers and cannot see buffer sizes);
buffers of the right size go through to the library. CPU only: the plan is a
stand-in with the fields the checks read and a null handle, so a call that
passes the checks ends in the library's own EINVAL for the null plan."""
import types

import numpy as np
import pytest

import paper_1502_05037_gb300 as pk
from paper_1502_05037_gb300 import _lib
from paper_1502_05037_gb300 import build as pbuild

NX = NY = 8
M, Q, R = 10, 9, 2


@pytest.fixture(scope="module")
def plan():
    pbuild.build()
    _lib.load()
    info = types.SimpleNamespace(N=NX * NY, M=M, D=Q * NX * NY, Kx=2 * NX, Ky=2 * NY, R=R, q=Q)
    return types.SimpleNamespace(handle=None, dtype=pk.PURIFY_F32, info=info)


def real(n, dt=np.float32):
    return np.zeros(n, dtype=dt)


def cplx(n, dt=np.complex64):
    return np.zeros(n, dtype=dt)


def calls(plan, x=None, y=None, xc=None, c=None, grid=None, w=None, eps=None):
    x = real(NX * NY) if x is None else x
    y = cplx(M) if y is None else y
    xc = cplx(NX * NY) if xc is None else xc
    c = real(Q * NX * NY) if c is None else c
    grid = cplx(4 * NX * NY) if grid is None else grid
    eps = np.ones(R) if eps is None else eps
    return [
        lambda: pk.purify_phi(plan, x, y),
        lambda: pk.purify_phi_adj(plan, y, xc),
        lambda: pk.purify_phi_normal(plan, x, x.copy()),
        lambda: pk.purify_fft2(plan, grid),
        lambda: pk.purify_psi(plan, c, x),
        lambda: pk.purify_psi_adj(plan, x, c),
        lambda: pk.purify_sdmm_solve(plan, y, eps, x, w=w, max_iter=1),
        lambda: pk.purify_pd_solve(plan, y, eps, x, w=w, iters=1),
        lambda: pk.purify_reweight(plan, x, 1.0, c),
        lambda: pk.purify_coef_std(plan, x),
    ]


def test_right_sizes_reach_the_library(plan):
    for f in calls(plan):
        with pytest.raises(pk.PurifyError) as e:
            f()
        assert e.value.status == _lib.PURIFY_EINVAL   # the null plan, rejected by the C side


@pytest.mark.parametrize("short", ["x", "y", "xc", "c", "grid", "eps"])
def test_short_buffers_are_refused(plan, short):
    kw = {"x": real(NX * NY - 1), "y": cplx(M - 1), "xc": real(2 * NX * NY - 1), "c": real(Q * NX * NY - 1),
          "grid": cplx(4 * NX * NY - 1), "eps": np.ones(R - 1)}
    refused = 0
    for f in calls(plan, **{short: kw[short]}):
        try:
            f()
        except ValueError:
            refused += 1
        except pk.PurifyError:
            pass
    # every call that takes that buffer refuses it
    want = {"x": 8, "y": 4, "xc": 1, "c": 3, "grid": 1, "eps": 2}[short]
    assert refused == want


def test_complex_output_of_the_adjoint_needs_two_values_per_pixel(plan):
    with pytest.raises(ValueError):
        pk.purify_phi_adj(plan, cplx(M), real(NX * NY))


def test_fp64_plans_need_eight_byte_values(plan):
    p64 = types.SimpleNamespace(handle=None, dtype=pk.PURIFY_F64, info=plan.info)
    with pytest.raises(ValueError):
        pk.purify_phi(p64, real(NX * NY), cplx(M, np.complex128))
    with pytest.raises(pk.PurifyError):
        pk.purify_phi(p64, real(NX * NY, np.float64), cplx(M, np.complex128))


def test_weights_are_checked(plan):
    with pytest.raises(ValueError):
        pk.purify_sdmm_solve(plan, cplx(M), np.ones(R), real(NX * NY), w=real(Q * NX * NY - 1), max_iter=1)
