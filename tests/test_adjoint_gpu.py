"""GPU parity of the adjoint (reverse-mode) path through the C ABI.

The CUDA pull-back of one step and of a checkpointed run is compared with the oracle's on the
same seeded inputs (FP64, element by element, relative L2), with the library's own forward map
by central finite differences, and with properties that hold at any size: the qubit norm is
conserved by every step, so for L = |x_n|^2 / 2 the gradient is exactly x_0 and dL/dg = 0; and a
phase-invariant loss has a gradient orthogonal to i x_0.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import objectives_ref
import oracle
from paper_1907_12834_gb300 import inputs, qlga

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


CASES = [  # (ndim, nx, ny, g, variant)
    (1, 200, 1, (1.0, -0.5, 0.2), 0),
    (1, 131, 1, (1.0, 0.8, -0.6), 1),
    (2, 40, 36, (1.0, 0.1, 1.0), 0),
    (2, 33, 20, (0.7, -0.4, 0.9), 1),
]


@pytest.mark.parametrize("ndim,nx,ny,g,variant", CASES)
def test_adjoint_step_matches_oracle(ndim, nx, ny, g, variant):
    rng = np.random.default_rng(100 + nx)
    x = 0.15 * rng.standard_normal((5, ny, nx, 2, 2))  # beta = ||delta W|| stays below 4
    w = rng.standard_normal((5, ny, nx, 2, 2))
    cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
    ref = w.copy()
    dref = oracle.vjp_step(x, ref, cfg)
    with qlga.Lattice(ndim, nx, ny, 64, g, kinetic_variant=variant) as lat:
        cot, d = lat.adjoint_step(_dev(x), _dev(w))
    assert _rel(cot.cpu().numpy(), ref) < FP64_TOL
    assert np.abs(d - dref).max() / np.abs(dref).max() < 1e-10


@pytest.mark.parametrize("ndim,nx,ny,g,variant", CASES[::2])
def test_adjoint_step_fp32_vs_oracle(ndim, nx, ny, g, variant):
    rng = np.random.default_rng(7 + nx)
    x = (0.1 * rng.standard_normal((5, ny, nx, 2, 2))).astype(np.float32).astype(np.float64)
    w = rng.standard_normal((5, ny, nx, 2, 2)).astype(np.float32).astype(np.float64)
    cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
    ref = w.copy()
    dref = oracle.vjp_step(x, ref, cfg)
    with qlga.Lattice(ndim, nx, ny, 32, g, kinetic_variant=variant) as lat:
        cot, d = lat.adjoint_step(_dev(x, torch.float32), _dev(w, torch.float32))
    assert _rel(cot.cpu().numpy(), ref) < 1e-5
    assert np.abs(d - dref).max() / np.abs(dref).max() < 1e-4


@pytest.mark.parametrize("ndim,nx,ny,g,variant,n,C", [
    (1, 64, 1, (1.0, -0.5, 0.2), 0, 25, 7),
    (1, 50, 1, (1.0, 0.8, -0.6), 1, 9, 20),
    (2, 24, 20, (1.0, 0.1, 1.0), 0, 12, 5),
    (2, 17, 16, (0.7, -0.4, 0.9), 1, 6, 1),
])
def test_adjoint_run_matches_oracle(ndim, nx, ny, g, variant, n, C):
    rng = np.random.default_rng(200 + n)
    x0 = 0.15 * rng.standard_normal((5, ny, nx, 2, 2))
    w = rng.standard_normal((5, ny, nx, 2, 2))
    cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
    ref = w.copy()
    dref = oracle.vjp_run(x0, n, ref, cfg)
    with qlga.Lattice(ndim, nx, ny, 64, g, kinetic_variant=variant) as lat:
        cot, d = lat.gradient(_dev(x0), n, _dev(w), checkpoint_every=C)
        xn = lat.get_state()
    xref = oracle.step(x0.copy(), cfg, n)
    assert _rel(xn, xref) < FP64_TOL            # the handle ends holding x_n
    assert _rel(cot.cpu().numpy(), ref) < 1e-10
    assert np.abs(d - dref).max() / np.abs(dref).max() < 1e-9


def test_adjoint_matches_finite_differences_fp64():
    """<dL/dx0, v> against the fourth-order central difference of the library's own forward map,
    L = <w, x_n>, on a small vortex-dipole state."""
    n, steps = 32, 40
    w4 = inputs.config4(n=n, separation=12, dtype=np.float64)
    rng = np.random.default_rng(3)
    x0 = w4.state
    v = rng.standard_normal(x0.shape) * 0.05
    w = rng.standard_normal(x0.shape)
    with qlga.Lattice(2, n, n, 64, w4.g) as lat:
        cot, _ = lat.gradient(_dev(x0), steps, _dev(w), checkpoint_every=16)

        def L(x):
            lat.load_state(_dev(x))
            lat.step(steps)
            return float(np.sum(w * lat.get_state()))

        h = 1e-5
        d1 = (L(x0 + h * v) - L(x0 - h * v)) / (2 * h)
        d2 = (L(x0 + 2 * h * v) - L(x0 - 2 * h * v)) / (4 * h)
        fd = (4 * d1 - d2) / 3
    ad = float(np.sum(cot.cpu().numpy() * v))
    assert abs(ad - fd) / abs(fd) < 1e-7


@pytest.mark.parametrize("precision,n,steps,C,tol", [
    (64, 512, 200, 100, 1e-10),
    (32, 512, 200, 100, 1e-4),
])
def test_norm_loss_gradient_is_x0_full_size(precision, n, steps, C, tol):
    """Config 4 lattice (512^2): every step conserves the qubit norm, so L = |x_n|^2 / 2 has
    dL/dx0 = x0 exactly and dL/dg = 0, along any trajectory.  Rounding in the pull-back is
    amplified like a perturbation of the forward run (the vortex background is dynamically
    unstable), so the check uses 200 steps."""
    dt = torch.float32 if precision == 32 else torch.float64
    w4 = inputs.config4(n=n, dtype=np.float32 if precision == 32 else np.float64)
    x0 = _dev(w4.state, dt)
    with qlga.Lattice(2, n, n, precision, w4.g) as lat:
        ws = lat.adjoint_workspace(steps, C)
        lat.adjoint_forward(x0, steps, C, ws)
        xn = lat.device_state()
        cot, d = lat.adjoint_backward(xn, steps, C, ws)
    err = float(torch.linalg.vector_norm((cot - x0).double()) / torch.linalg.vector_norm(x0.double()))
    assert err < tol
    norm2 = float((x0.double() ** 2).sum())
    assert np.abs(d).max() / norm2 < (1e-9 if precision == 64 else 1e-3)


def test_phase_invariant_loss_gradient_orthogonal_to_gauge_direction():
    """A loss invariant under x -> e^{i alpha} x (the dynamics commute with the global phase) has
    <dL/dx0, i x0> = 0; checked for the m_f = 0 population and the singlet fraction."""
    n, steps = 48, 60
    w4 = inputs.config4(n=n, separation=16, dtype=np.float64)
    x0 = _dev(w4.state).requires_grad_(True)
    g = torch.tensor(w4.g, dtype=torch.float64, device="cuda")
    xn = qlga.evolve(x0, g, steps, checkpoint_every=25)
    loss = qlga.population(xn, 2) + qlga.singlet_fraction(xn)
    (gx,) = torch.autograd.grad(loss, x0)
    ix = torch.stack([-x0[..., 1], x0[..., 0]], dim=-1).detach()  # i x0 in (re, im) pairs
    dot = float((gx * ix).sum())
    assert abs(dot) / (float(gx.norm()) * float(ix.norm())) < 1e-10


def _objective_params_case():
    n, steps, sep = 40, 80, 14
    w4 = inputs.config4(n=n, separation=sep, dtype=np.float64)
    psi = inputs.state_to_boson(w4.state) / w4.eps
    cores = inputs.dipole_cores(n, n, sep, "a")
    return n, steps, w4, psi, cores


def test_objective_gradients_match_finite_differences():
    """Gradients of (m_f = 0 population + singlet fraction) after 80 steps with respect to the
    vortex velocities (windowed local kicks), a relative phase and the couplings g1, g2, against
    fourth-order central differences of the same forward runs (h = 1e-5)."""
    n, steps, w4, psi, cores = _objective_params_case()
    dev = "cuda"

    def loss_of(vel, ph, g):
        x0 = inputs.kicked_state(psi, w4.eps, cores, vel, (4,), ph)
        xn = qlga.evolve(x0, g, steps, checkpoint_every=20)
        return qlga.population(xn, 2) * 1e3 + qlga.singlet_fraction(xn)

    vel = torch.full((len(cores), 2), 0.02, dtype=torch.float64, device=dev)
    vel[1] *= -1
    ph = torch.tensor([0.3], dtype=torch.float64, device=dev)
    g = torch.tensor(w4.g, dtype=torch.float64, device=dev)
    vel.requires_grad_(True)
    ph.requires_grad_(True)
    g.requires_grad_(True)
    L = loss_of(vel, ph, g)
    gv, gp, gg = torch.autograd.grad(L, (vel, ph, g))

    def fd(which, idx, h=1e-5):
        def at(delta):
            v2, p2, g2 = vel.detach().clone(), ph.detach().clone(), g.detach().clone()
            {"v": v2, "p": p2, "g": g2}[which].view(-1)[idx] += delta
            with torch.no_grad():
                return float(loss_of(v2, p2, g2))
        d1 = (at(h) - at(-h)) / (2 * h)
        d2 = (at(2 * h) - at(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    checks = [("v", 0, gv.view(-1)[0]), ("v", 3, gv.view(-1)[3]), ("p", 0, gp[0]),
              ("g", 1, gg[1]), ("g", 2, gg[2])]
    for which, idx, ad in checks:
        ref = fd(which, idx)
        assert abs(float(ad) - ref) <= 1e-6 * max(abs(ref), 1e-3), (which, idx, float(ad), ref)


def test_objective_gradient_matches_oracle():
    """dL/dx0 of (m_f = 0 population + singlet fraction) after 30 steps: CUDA adjoint through
    the autograd function against the oracle's pull-back of the same cotangent."""
    n, steps, sep = 24, 30, 10
    w4 = inputs.config4(n=n, separation=sep, dtype=np.float64)
    x0 = np.ascontiguousarray(w4.state)
    cfg = oracle.make_cfg(2, n, n, *w4.g)
    xn_ref = oracle.step(x0.copy(), cfg, steps)
    xt = torch.tensor(xn_ref, requires_grad=True)
    lref = objectives_ref.population(xt, 2) + objectives_ref.singlet_fraction(xt)
    (cot_n,) = torch.autograd.grad(lref, xt)
    ref = cot_n.numpy().copy()
    dref = oracle.vjp_run(x0, steps, ref, cfg)

    x0d = _dev(x0).requires_grad_(True)
    g = torch.tensor(w4.g, dtype=torch.float64, device="cuda", requires_grad=True)
    xn = qlga.evolve(x0d, g, steps, checkpoint_every=8)
    L = qlga.population(xn, 2) + qlga.singlet_fraction(xn)
    gx, gg = torch.autograd.grad(L, (x0d, g))
    assert _rel(gx.cpu().numpy(), ref) < 1e-10
    assert np.abs(gg.cpu().numpy() - dref).max() / np.abs(dref).max() < 1e-9


def test_autograd_gradcheck_small():
    rng = np.random.default_rng(9)
    x0 = _dev(0.2 * rng.standard_normal((5, 1, 8, 2, 2))).requires_grad_(True)
    g = torch.tensor([1.0, -0.5, 0.2], dtype=torch.float64, device="cuda", requires_grad=True)
    w = _dev(rng.standard_normal((5, 1, 8, 2, 2)))

    def f(x, gg):
        return (qlga.evolve(x, gg, 3, checkpoint_every=2) * w).sum()

    assert torch.autograd.gradcheck(f, (x0, g), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)


def test_fp32_gradient_tracks_fp64():
    n, steps = 64, 100
    w4 = inputs.config4(n=n, separation=20, dtype=np.float64)
    grads = {}
    for dt in (torch.float64, torch.float32):
        x0 = _dev(w4.state, dt).requires_grad_(True)
        g = torch.tensor(w4.g, dtype=torch.float64, device="cuda")
        xn = qlga.evolve(x0, g, steps, checkpoint_every=30)
        L = qlga.population(xn.double(), 2) * 1e3 + qlga.singlet_fraction(xn.double())
        (gx,) = torch.autograd.grad(L, x0)
        grads[dt] = gx.double().cpu().numpy()
    assert _rel(grads[torch.float32], grads[torch.float64]) < 1e-3


def test_adjoint_edge_cases():
    rng = np.random.default_rng(4)
    x0 = 0.1 * rng.standard_normal((5, 1, 16, 2, 2))
    w = rng.standard_normal(x0.shape)
    with qlga.Lattice(1, 16, 1, 64, (1.0, 0.3, 0.2)) as lat:
        cot, d = lat.gradient(_dev(x0), 0, _dev(w), checkpoint_every=5)   # no steps: identity
        assert np.array_equal(cot.cpu().numpy(), w) and not np.any(d)
        cot1, d1 = lat.gradient(_dev(x0), 1, _dev(w), checkpoint_every=1)
        cot2, d2 = lat.adjoint_step(_dev(x0), _dev(w))
        assert _rel(cot1.cpu().numpy(), cot2.cpu().numpy()) < 1e-15 and np.allclose(d1, d2, rtol=1e-14)
        buf, nb = lat.adjoint_workspace(10, 3)
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_adjoint_forward(lat.handle, _dev(x0).data_ptr(), 10, 3, lat._aligned(buf), nb - 256)
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
    with qlga.Lattice(1, 16, 1, 64, (1.0, 0.3, 0.2), interleave=1) as lat:
        with pytest.raises(qlga.QlgaError) as e:
            lat.adjoint_step(_dev(x0), _dev(w))
        assert e.value.status == qlga.QLGA_ERR_UNSUPPORTED


def test_config4_objective_gradients_fp64_full_lattice():
    """Config 4 lattice (512^2, FP64, 100 steps, checkpoints every 50): gradients of the final
    m_f = 0 population and singlet fraction with respect to the 4 velocity components of the
    vortex pair in m = +2, the 2 local phases of the pair and g1, g2, against fourth-order central
    differences (h = 1e-5), to 1e-5 relative.  The global phases of the occupied levels m = +2 and
    m = -2 are symmetry directions of this loss (global phase, rotation about z): their gradients
    must vanish.  (Over the full 2000 steps the dynamics amplify rounding beyond any
    finite-difference check; see the norm-identity test.)"""
    n, steps = 512, 100
    w4 = inputs.config4(n=n, dtype=np.float64)
    psi = inputs.state_to_boson(w4.state) / w4.eps
    cores = inputs.dipole_cores(n, n, 64.0, "a")[:2]      # vortex and antivortex of m = +2

    def loss_of(vel, cph, lph, g):
        x0 = inputs.kicked_state(psi, w4.eps, cores, vel, (0, 4), lph, core_phases=cph)
        xn = qlga.evolve(x0, g, steps, checkpoint_every=50)
        return qlga.population(xn, 2) * 1e2 + qlga.singlet_fraction(xn)

    dev = "cuda"
    vel = torch.tensor([[0.01, 0.0], [-0.01, 0.0]], dtype=torch.float64, device=dev, requires_grad=True)
    cph = torch.tensor([0.3, -0.2], dtype=torch.float64, device=dev, requires_grad=True)
    lph = torch.tensor([0.2, -0.1], dtype=torch.float64, device=dev, requires_grad=True)
    g = torch.tensor(w4.g, dtype=torch.float64, device=dev, requires_grad=True)
    gv, gc, gl, gg = torch.autograd.grad(loss_of(vel, cph, lph, g), (vel, cph, lph, g))
    scale = max(float(gv.abs().max()), float(gc.abs().max()), float(gg.abs().max()))
    assert float(gl.abs().max()) <= 1e-9 * scale

    def fd(which, idx, h=1e-5):
        def at(delta):
            p = {"v": vel.detach().clone(), "c": cph.detach().clone(), "g": g.detach().clone()}
            p[which].view(-1)[idx] += delta
            with torch.no_grad():
                return float(loss_of(p["v"], p["c"], lph.detach(), p["g"]))
        d1 = (at(h) - at(-h)) / (2 * h)
        d2 = (at(2 * h) - at(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    checks = [("v", i, gv.view(-1)[i]) for i in range(4)] + [("c", i, gc[i]) for i in range(2)] + \
             [("g", 1, gg[1]), ("g", 2, gg[2])]
    for which, idx, ad in checks:
        ref = fd(which, idx)
        assert abs(float(ad) - ref) <= 1e-5 * max(abs(ref), 1e-3 * scale), (which, idx, float(ad), ref)


def test_energy_objective_gradient_1d_fp64():
    """Breather-type objective: the energy of the final boson field (the library's energy
    observable, written in torch and checked against the oracle's) after 300 steps of a kicked
    two-soliton state (L = 2048, FP64), differentiated through the adjoint with respect to the
    initial state (along a random direction) and the couplings g1, g2 of the dynamics, against
    fourth-order central differences."""
    L, steps = 2048, 300
    w = inputs.config1(L=L, precision=64)
    g_eval = w.g
    x0 = _dev(w.state).requires_grad_(True)
    g = torch.tensor(w.g, dtype=torch.float64, device="cuda", requires_grad=True)
    cfg = oracle.make_cfg(1, L, 1, *w.g)
    e_oracle = oracle.observables(np.ascontiguousarray(w.state), cfg)["energy"]
    assert abs(float(qlga.energy(x0.detach(), g_eval)) - e_oracle) <= 1e-12 * abs(e_oracle)

    def loss(x, gg):
        return qlga.energy(qlga.evolve(x, gg, steps, checkpoint_every=64), g_eval)

    gx, gg = torch.autograd.grad(loss(x0, g), (x0, g))
    rng = np.random.default_rng(12)
    v = _dev(rng.standard_normal(w.state.shape) * 1e-2)

    def fd(fun, h):
        d1 = (fun(h) - fun(-h)) / (2 * h)
        d2 = (fun(2 * h) - fun(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    with torch.no_grad():
        ref_x = fd(lambda h: float(loss(x0.detach() + h * v, g.detach())), 1e-4)
        ad_x = float((gx * v).sum())
        assert abs(ad_x - ref_x) <= 1e-6 * abs(ref_x)
        for i in (1, 2):
            e = torch.zeros(3, dtype=torch.float64, device="cuda")
            e[i] = 1.0
            ref = fd(lambda h: float(loss(x0.detach(), g.detach() + h * e)), 1e-5)
            # a floor at the finite differences' own rounding (g2 does not enter when the singlet
            # amplitude of the state vanishes, as for these soliton rows)
            scale = max(abs(float(gg[1])), abs(ad_x))
            assert abs(float(gg[i]) - ref) <= 1e-6 * abs(ref) + 1e-8 * scale, (i, float(gg[i]), ref)
