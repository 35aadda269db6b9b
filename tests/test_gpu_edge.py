"""Edge cases of the float64 path through the C ABI: the smallest inputs, an
iteration cap that stops the solve early (the partial iterate must equal the
oracle's PCG iterate after the same number of steps), a zero right-hand side,
bitwise reproducibility of T*v (integer accumulation of the reciprocal
grid, fixed-order sums elsewhere), and atoms on the cell faces of the
neighbour search and on the box faces."""
import numpy as np
import pytest

from oracle import Setup
from oracle.setup import DEBYE
from oracle.solver import Operator, pcg
from paper_1906_01211_gb300.synth import WATER_648, System, make_waters
from tests.parity_metrics import assert_fields

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def solver(w, max_iter=100, tol=None):
    from paper_1906_01211_gb300 import amoebapol as ap
    return ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                     tol_debye=tol or w.tol_debye, max_iter=max_iter))


def test_one_atom_is_rejected():
    from paper_1906_01211_gb300 import amoebapol as ap
    w = WATER_648
    s = solver(w)
    one = w.system()
    sub = System(xyz=one.xyz[:1], q=one.q[:1], dip=one.dip[:1], quad=one.quad[:1], alpha=one.alpha[:1],
                 thole=one.thole[:1], mol=one.mol[:1], box=one.box)
    with pytest.raises(ap.AmpError) as e:
        s.set_synthetic(sub)
    assert e.value.code == ap.AMP_ERR_ARG


@pytest.mark.parametrize("cap", [1, 2, 3])
def test_iteration_cap_returns_the_pcg_iterate(cap):
    from paper_1906_01211_gb300 import amoebapol as ap
    w = WATER_648
    sysm = w.system()
    setup = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=5)
    op = Operator(sysm, setup)
    E0 = op.permanent_field()
    mu_o, it_o, rms_o = pcg(op.apply_A, sysm.alpha, E0, w.tol_debye, max_iter=cap)
    assert it_o == cap
    s = solver(w, max_iter=cap)
    s.set_synthetic(sysm)
    E0g = s.permanent_field()
    with pytest.raises(ap.AmpError) as e:
        s.solve(E0g)
    assert e.value.code == ap.AMP_ERR_NOT_CONVERGED
    mu, it, rms = s.solve(E0g, check=False)
    assert it == cap
    d = mu.cpu().numpy() - mu_o
    assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-9
    assert abs(rms / rms_o - 1) < 1e-8


def test_zero_field_converges_at_once():
    w = WATER_648
    base = w.system()
    sysm = System(xyz=base.xyz, q=np.zeros_like(base.q), dip=np.zeros_like(base.dip),
                  quad=np.zeros_like(base.quad), alpha=base.alpha, thole=base.thole, mol=base.mol, box=base.box)
    s = solver(w)
    s.set_synthetic(sysm)
    E0 = s.permanent_field()
    assert float(torch.abs(E0).max()) == 0.0
    mu, it, rms = s.solve(E0)
    assert it == 0 and float(torch.abs(mu).max()) == 0.0


def test_two_atom_box_matches_oracle():
    L = 16.0
    base = make_waters(2, L, 3)
    sysm = System(xyz=base.xyz[:2], q=base.q[:2], dip=base.dip[:2], quad=base.quad[:2], alpha=base.alpha[:2],
                  thole=base.thole[:2], mol=base.mol[:2], box=L)
    setup = Setup(box=L, cutoff=7.0, beta=0.5446, grid=16, order=5)
    op = Operator(sysm, setup)
    from paper_1906_01211_gb300 import amoebapol as ap
    s = ap.Polarization(ap.Config(box=L, cutoff=7.0, ewald_beta=0.5446, pme_grid=16, tol_debye=1e-10))
    s.set_synthetic(sysm)
    E0 = s.permanent_field().cpu().numpy()
    # E0 (~4e-4) is what is left of parts of ~6e-2 (the excluded pair and the
    # reciprocal part), both float64 on the GPU: held to 1e-12 of E0 itself
    assert_fields(E0, op.permanent_field(), 1e-12)
    v = np.random.default_rng(2).normal(size=(2, 3))
    t = s.apply_T(torch.tensor(v)).cpu().numpy()
    assert_fields(t, op.apply_T(v), 1e-12)


def test_apply_T_is_bitwise_reproducible():
    w = WATER_648
    s = solver(w)
    s.set_synthetic(w.system())
    v = torch.tensor(np.random.default_rng(11).normal(size=(w.n_waters * 3, 3)) * 0.1)
    a = s.apply_T(v).clone()
    b = s.apply_T(v).clone()
    assert torch.equal(a, b)


def test_list_refill_paths_on_one_context():
    """One context through every neighbour-list fill path: the first call
    sizes the lists; later calls fill them before the counts reach the host
    and refill on the two-pass path when the lists outgrow their buffers
    (twice the waters in the same box) or an owned row overflows its slab
    row (waters packed into one corner), alone or together. Pair count, E0 and T*v against the
    oracle after each call."""
    from paper_1906_01211_gb300 import amoebapol as ap
    from paper_1906_01211_gb300.synth import System, density_box_edge, make_waters
    L = density_box_edge(300)
    rc, beta = 7.0, 0.5446
    K = 32
    s = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=1e-10))
    sparse = make_waters(150, L, 71)
    dense = make_waters(300, L, 72)
    # two thirds of the dense waters squeezed into one corner (0.3 of the
    # edge): up to 345 owned neighbours per row there, the slab holds 288
    xyz = dense.xyz.copy()
    n_c = 3 * 200
    xyz[:n_c] = xyz[:n_c] * 0.3
    packed = System(xyz=xyz, q=dense.q, dip=dense.dip, quad=dense.quad, alpha=dense.alpha, thole=dense.thole,
                    mol=dense.mol, box=L)
    rng = np.random.default_rng(73)
    # sparse sizes the lists; dense outgrows them; packed outgrows them and
    # overflows a slab row; sparse and dense then fit; packed again fits but
    # overflows a slab row
    for sysm in (sparse, dense, packed, sparse, dense, packed):
        op = Operator(sysm, Setup(box=L, cutoff=rc, beta=beta, grid=K, order=5))
        s.set_synthetic(sysm)
        assert s.pair_count() == op.n_pairs
        E0 = s.permanent_field().cpu().numpy()
        assert np.linalg.norm(E0 - op.permanent_field()) < 1e-12 * np.linalg.norm(op.permanent_field())
        v = rng.normal(size=(sysm.n, 3)) * 0.1
        t = s.apply_T(torch.tensor(v)).cpu().numpy()
        ref = op.apply_T(v)
        assert np.linalg.norm(t - ref) < 1e-12 * np.linalg.norm(ref)
    s.close()


def test_atoms_on_cell_faces_and_box_edges():
    """Oxygens exactly on the cell lattice of the neighbour search (seven
    cells per axis, so each atom's candidate runs are trimmed to the cells
    within reach of it), on the box's faces at 0 and some moved by one box
    edge (-L or +L) out of the box: every pair within the cutoff must still be
    found, with the oracle's pair count, field, T*v and dipoles."""
    from oracle.solver import solve
    from paper_1906_01211_gb300.synth import small_box_settings
    nc = 7
    L = 26.2345
    h = L / nc
    rc, beta, K = small_box_settings(L)
    assert int(np.floor(2.0 * L / rc)) == nc
    base = make_waters(nc ** 3, L, 17)
    rng = np.random.default_rng(17)
    ijk = np.stack(np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij"), -1).reshape(-1, 3)
    target = ijk * h
    image = np.zeros_like(target)
    pick = rng.random(len(target)) < 0.3
    axis = rng.integers(0, 3, len(target))
    image[pick, axis[pick]] = rng.choice([-L, L], pick.sum())
    shift = np.repeat(target + image - base.xyz[0::3], 3, axis=0)
    sysm = System(xyz=base.xyz + shift, q=base.q, dip=base.dip, quad=base.quad, alpha=base.alpha,
                  thole=base.thole, mol=base.mol, box=L)
    setup = Setup(box=L, cutoff=rc, beta=beta, grid=K, order=5)
    op = Operator(sysm, setup)
    from paper_1906_01211_gb300 import amoebapol as ap
    s = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=1e-10))
    s.set_synthetic(sysm)
    assert s.pair_count() == op.n_pairs
    E0 = s.permanent_field()
    assert_fields(E0.cpu().numpy(), op.permanent_field(), 1e-12)
    v = np.random.default_rng(3).normal(size=(sysm.n, 3)) * 0.1
    assert_fields(s.apply_T(torch.tensor(v)).cpu().numpy(), op.apply_T(v), 1e-12)
    mu, it, rms = s.solve(E0)
    mu_ref, it_ref, _ = solve(op, op.permanent_field(), 1e-10)
    assert it == it_ref
    d = mu.cpu().numpy() - mu_ref
    assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-8


def test_energy_on_device_matches_host_energy():
    """The binding's energy_on_device (the allocation-free energy call, on the
    context's stream, result left on the device) gives the context's energy,
    up to the order of the two reductions."""
    w = WATER_648
    s = solver(w)
    s.set_synthetic(w.system())
    E0 = s.permanent_field()
    mu, _, _ = s.solve(E0)
    U = s.energy(mu, E0)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    s.energy_on_device(mu, E0, out)
    torch.cuda.synchronize()
    assert abs(out.item() / U - 1.0) < 1e-12
