"""Neighbour-list reuse with a skin (amp_set_list_skin / amp_update_positions)
through the C ABI, against the CPU oracle on the moved positions: the lists
filtered out of the stored candidates give the same pairs as a new cell
search, and E0, T*v, the induced dipoles and the energy match the oracle at
the float64 tolerances; a move beyond skin/2 is refused and changes nothing."""
import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.setup import DEBYE
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import WATER_648, System, density_box_edge, make_waters

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def moved(sysm, xyz):
    return System(xyz=xyz, q=sysm.q, dip=sysm.dip, quad=sysm.quad, alpha=sysm.alpha, thole=sysm.thole,
                  mol=sysm.mol, box=sysm.box)


def ball(rng, n, radius):
    """n displacements uniform in a ball of the given radius."""
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * radius * rng.uniform(size=(n, 1)) ** (1.0 / 3.0)


def solver(L, rc, beta, K, tol, precision="fp64"):
    from paper_1906_01211_gb300 import amoebapol as ap
    return ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=tol,
                                     precision=precision))


def check_against_oracle(s, sysm, setup, tol, rng):
    op = Operator(sysm, setup)
    assert s.pair_count() == op.n_pairs
    E0 = s.permanent_field().cpu().numpy()
    E0_ref = op.permanent_field()
    assert rel(E0, E0_ref) < 1e-12
    v = rng.normal(size=(sysm.n, 3)) * 0.1
    assert rel(s.apply_T(torch.tensor(v)).cpu().numpy(), op.apply_T(v)) < 1e-12
    mu, it, rms = s.solve(torch.tensor(E0))
    mu_ref, it_ref, _ = solve(op, E0_ref, tol)
    d = mu.cpu().numpy() - mu_ref
    assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-8
    U = s.energy(mu, torch.tensor(E0))
    assert abs(U / polarization_energy(mu_ref, E0_ref) - 1) < 1e-10
    return E0


def test_update_within_half_skin_matches_the_oracle():
    w = WATER_648
    skin = 1.0
    setup = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=5)
    rng = np.random.default_rng(81)
    s = solver(w.L, w.cutoff, w.beta, w.grid, 1e-10)
    s.set_list_skin(skin)
    sys0 = w.system()
    s.set_synthetic(sys0)
    check_against_oracle(s, sys0, setup, 1e-10, rng)
    # two moves of up to 0.2 A each: at most 0.4 A from the positions of set_system
    sys1 = moved(sys0, sys0.xyz + ball(rng, sys0.n, 0.2))
    assert s.update_positions(sys1.xyz)
    E0_1 = check_against_oracle(s, sys1, setup, 1e-10, rng)
    sys2 = moved(sys1, sys1.xyz + ball(rng, sys0.n, 0.2))
    assert s.update_positions(sys2.xyz)
    check_against_oracle(s, sys2, setup, 1e-10, rng)
    # a fresh context without a skin on the same positions: the same pairs
    f = solver(w.L, w.cutoff, w.beta, w.grid, 1e-10)
    f.set_synthetic(sys2)
    assert f.pair_count() == s.pair_count()
    assert rel(s.permanent_field().cpu().numpy(), f.permanent_field().cpu().numpy()) < 1e-13
    f.close()
    # one atom 0.6 A from where set_system saw it: refused, nothing changes
    xyz3 = sys0.xyz.copy()
    xyz3[7] += np.array([0.6, 0.0, 0.0])
    assert not s.update_positions(xyz3)
    E0_still = s.permanent_field().cpu().numpy()
    E0_2 = Operator(sys2, setup).permanent_field()
    assert rel(E0_still, E0_2) < 1e-12
    # a new set_system there re-arms the reuse
    sys3 = moved(sys0, xyz3)
    s.set_synthetic(sys3)
    assert s.update_positions(sys3.xyz + ball(rng, sys0.n, 0.1))
    s.close()
    assert np.isfinite(E0_1).all()


def test_update_mixed_precision_and_periodic_wrap():
    """Mixed precision on a box whose atoms cross the periodic boundary
    between set_system and the update."""
    nw = 300
    L = density_box_edge(nw)
    rc, beta, K = 7.0, 0.5446, 32
    skin = 0.8
    setup = Setup(box=L, cutoff=rc, beta=beta, grid=K, order=5)
    rng = np.random.default_rng(82)
    sys0 = make_waters(nw, L, 83)
    s = solver(L, rc, beta, K, 1e-6, precision="mixed")
    s.set_list_skin(skin)
    s.set_synthetic(sys0)
    # shift everything by almost L along x plus a small jitter: positions wrap
    sys1 = moved(sys0, sys0.xyz + np.array([L - 0.1, 0.0, 0.0]) + ball(rng, sys0.n, 0.25))
    assert s.update_positions(sys1.xyz)
    op = Operator(sys1, setup)
    assert s.pair_count() == op.n_pairs
    E0 = s.permanent_field()
    mu, it, rms = s.solve(E0)
    mu_ref, _, _ = solve(op, op.permanent_field(), 1e-10)
    d = mu.cpu().numpy() - mu_ref
    assert DEBYE * np.sqrt((d * d).sum() / sys1.n) < 1e-5
    s.close()


def test_skin_arguments_are_checked():
    from paper_1906_01211_gb300 import amoebapol as ap
    w = WATER_648
    s = solver(w.L, w.cutoff, w.beta, w.grid, 1e-8)
    for bad in (-0.5, w.L / 2.0 - w.cutoff):  # negative; cutoff + skin = box/2
        with pytest.raises(ap.AmpError) as e:
            s.set_list_skin(bad)
        assert e.value.code == ap.AMP_ERR_ARG
    s.set_synthetic(w.system())
    # no skin at set_system: every update is refused
    assert not s.update_positions(w.system().xyz)
    s.close()


def test_predictor_of_a_repeated_solution_starts_converged():
    """The ASPC coefficients sum to one: with the same system solved k + 2
    times the predicted start is the solution, and the next solve takes no
    iteration; before the history is full the start is alpha*E0."""
    w = WATER_648
    s = solver(w.L, w.cutoff, w.beta, w.grid, 1e-8)
    sysm = w.system()
    s.set_synthetic(sysm)
    s.set_predictor(1)  # three solutions: 2.5 mu_-1 - 2 mu_-2 + 0.5 mu_-3
    E0 = s.permanent_field()
    mu_cold, it_cold, _ = s.solve(E0)
    mu1, it1, _ = s.solve(E0, predict=True)  # history 1 < 3: cold start again
    assert it1 == it_cold
    s.solve(E0, predict=True)
    mu3, it3, _ = s.solve(E0, predict=True)  # history 3: predicted = mu
    assert it3 == 0
    d = (mu3 - mu_cold).cpu().numpy()
    assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-8
    # a new system clears the history
    s.set_synthetic(sysm)
    E0 = s.permanent_field()
    _, it4, _ = s.solve(E0, predict=True)
    assert it4 == it_cold
    s.close()


def test_predictor_along_a_trajectory_matches_the_oracle():
    """Frames of a random walk through list reuse, each solved from the
    predictor (order 0 = linear extrapolation once two solutions exist):
    every frame converges to the oracle's dipoles, in fewer iterations than a
    cold start once the history is full."""
    from paper_1906_01211_gb300 import amoebapol as ap
    w = WATER_648
    setup = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=5)
    rng = np.random.default_rng(91)
    s = solver(w.L, w.cutoff, w.beta, w.grid, 1e-8)
    s.set_list_skin(1.0)
    s.set_predictor(0)
    sysm = w.system()
    s.set_synthetic(sysm)
    xyz = sysm.xyz.copy()
    iters = []
    for f in range(5):
        if f:
            xyz = xyz + rng.normal(size=xyz.shape) * 0.01
            assert s.update_positions(xyz)
        E0 = s.permanent_field()
        mu, it, _ = s.solve(E0, predict=True)
        iters.append(it)
        op = Operator(moved(sysm, xyz), setup)
        mu_ref, it_ref, _ = solve(op, op.permanent_field(), 1e-8)
        d = mu.cpu().numpy() - mu_ref
        assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-7
    assert max(iters[2:]) < iters[0]
    with pytest.raises(ap.AmpError):
        s.set_predictor(7)
    s.close()
