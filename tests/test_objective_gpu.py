"""The objectives that gradients are taken of, computed by the library (qlga_objective): the
population of one level, the singlet fraction and the energy (Sec. III.B Eq. cmap; the energy
functional of Eq. eomspin2 with forward differences), with their cotangents.

Values against the FP64 oracle's observables of the same state (1e-12 in FP64); cotangents and
the energy's coupling derivatives against PyTorch autograd of the plain formulas
(tests/objectives_ref.py) in FP64 on the CPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import objectives_ref as R  # noqa: E402
import oracle  # noqa: E402
from paper_1907_12834_gb300 import inputs as I  # noqa: E402
from paper_1907_12834_gb300 import qlga  # noqa: E402

G = (1.0, 0.8, -0.6)


def _ref_grads(st, g, level, w):
    x = torch.tensor(np.asarray(st, np.float64), requires_grad=True)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    vals = torch.stack([R.population(x, level), R.singlet_fraction(x), R.energy(x, gt)])
    L = (vals * torch.tensor(w, dtype=torch.float64)).sum()
    gx, gg = torch.autograd.grad(L, (x, gt))
    return vals.detach().numpy(), gx.numpy(), gg.numpy()


@pytest.mark.parametrize("precision,ndim,nx,ny,level", [(64, 1, 300, 1, 2), (64, 2, 37, 21, 2),
                                                        (64, 2, 64, 40, 0), (32, 2, 96, 33, 2),
                                                        (32, 1, 1000, 1, 4)])
def test_objective_values_and_cotangent(precision, ndim, nx, ny, level):
    rng = np.random.default_rng(nx * ny + level)
    st = I.random_state(rng, nx, ny, scale=0.1)
    if precision == 32:
        st = st.astype(np.float32)
    w = rng.standard_normal(3)
    vals_ref, gx_ref, gg_ref = _ref_grads(st, G, level, w)
    o = oracle.observables(np.asarray(st, np.float64), oracle.make_cfg(ndim, nx, ny, *G))
    assert vals_ref[0] == pytest.approx(o["pop"][level], rel=1e-12)        # the reference's own pins
    assert vals_ref[1] == pytest.approx(o["singlet_fraction"], rel=1e-12)
    assert vals_ref[2] == pytest.approx(o["energy"], rel=1e-12)

    dt = torch.float64 if precision == 64 else torch.float32
    x = torch.tensor(st, dtype=dt, device="cuda")
    with qlga.Lattice(ndim, nx, ny, precision=precision, g=G) as lat:
        cot = torch.empty_like(x)
        vals, dg = qlga.qlga_objective(lat.handle, x.data_ptr(), level, G, w, cot.data_ptr())
        vals_only, none = qlga.qlga_objective(lat.handle, x.data_ptr(), level, G)
    assert none is None and np.array_equal(vals, vals_only)
    tol = 1e-12 if precision == 64 else 2e-6
    np.testing.assert_allclose(vals, [o["pop"][level], o["singlet_fraction"], o["energy"]], rtol=tol)
    got = cot.double().cpu().numpy()
    ctol = 1e-12 if precision == 64 else 1e-5
    assert np.linalg.norm(got - gx_ref) <= ctol * np.linalg.norm(gx_ref)
    np.testing.assert_allclose(dg, gg_ref, rtol=tol, atol=tol * np.abs(gg_ref).max())


def test_objective_autograd_functions():
    rng = np.random.default_rng(3)
    st = I.random_state(rng, 48, 20, scale=0.1)
    x = torch.tensor(st, device="cuda", requires_grad=True)
    g = torch.tensor(G, dtype=torch.float64, device="cuda", requires_grad=True)
    L = 2.0 * qlga.population(x, 2) - 3.0 * qlga.singlet_fraction(x) + 0.5 * qlga.energy(x, g)
    gx, gg = torch.autograd.grad(L, (x, g))
    _, gx_ref, gg_ref = _ref_grads(st, G, 2, (2.0, -3.0, 0.5))
    assert np.linalg.norm(gx.cpu().numpy() - gx_ref) <= 1e-12 * np.linalg.norm(gx_ref)
    np.testing.assert_allclose(gg.cpu().numpy(), gg_ref, rtol=1e-12)
    with pytest.raises(TypeError):
        qlga.population(torch.tensor(st), 2)          # no CPU path: the library computes on the GPU


def test_objective_rejects_bad_arguments():
    with qlga.Lattice(2, 32, 16, precision=64, g=G) as lat:
        x = torch.zeros((5, 16, 32, 2, 2), dtype=torch.float64, device="cuda")
        cot = torch.empty_like(x)
        for args in ((5, G, None, 0), (-1, G, None, 0), (2, G, None, cot.data_ptr())):
            with pytest.raises(qlga.QlgaError) as e:
                qlga.qlga_objective(lat.handle, x.data_ptr(), *args)
            assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_objective(lat.handle, x.data_ptr(), 2, (1.0, float("nan"), 0.0))
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        vals, _ = qlga.qlga_objective(lat.handle, x.data_ptr(), 2, G)      # zero state: all zero
        assert not np.any(vals)
