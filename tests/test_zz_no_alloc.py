"""The allocation-free energy entry point against the context-based one.

amp_polarization_energy_noalloc serves callers that cannot allocate device
memory when they need the energy (a framework owning all device memory in its
own pool, or a loop that must avoid cudaMalloc's implicit synchronisation).
It keeps its partial sums in a fixed device array shared by every call, so
this test calls it twice in a row, on systems of different sizes, and checks
each result against amp_polarization_energy within the energy tolerance of
the other GPU tests. This file is collected last on purpose.
"""
import pytest

from paper_1906_01211_gb300.synth import WATER_648, WATER_23556

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def solved(w):
    from paper_1906_01211_gb300 import amoebapol as ap
    p = ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                  tol_debye=w.tol_debye))
    p.set_synthetic(w.system())
    E0 = p.permanent_field()
    mu, _, _ = p.solve(E0)
    return p, mu, E0


def test_noalloc_energy_matches_context_energy_twice_in_a_row():
    from paper_1906_01211_gb300 import amoebapol as ap
    stream = torch.cuda.current_stream().cuda_stream
    cases = [solved(WATER_23556), solved(WATER_648)]
    u_dev = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for k, (p, mu, E0) in enumerate(cases):
        code = ap.amp_polarization_energy_noalloc(mu.shape[0], mu.data_ptr(), E0.data_ptr(),
                                                  u_dev[k:k + 1].data_ptr(), stream)
        assert code == ap.AMP_OK
    torch.cuda.synchronize()
    for k, (p, mu, E0) in enumerate(cases):
        ref = p.energy(mu, E0)
        got = float(u_dev[k].item())
        assert abs(got / ref - 1.0) < 1e-10, (k, got, ref)


def test_noalloc_rejects_oversize_and_bad_arguments():
    from paper_1906_01211_gb300 import amoebapol as ap
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    u = torch.zeros((1,), dtype=torch.float64, device="cuda")
    big = ap.AMP_NOALLOC_MAX_ATOMS + 1
    assert ap.amp_polarization_energy_noalloc(big, x.data_ptr(), x.data_ptr(), u.data_ptr()) \
        == ap.AMP_ERR_TOO_LARGE
    assert ap.amp_polarization_energy_noalloc(0, x.data_ptr(), x.data_ptr(), u.data_ptr()) == ap.AMP_ERR_ARG
    assert ap.amp_polarization_energy_noalloc(4, 0, x.data_ptr(), u.data_ptr()) == ap.AMP_ERR_ARG
