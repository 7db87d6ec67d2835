"""The no-allocation collision entry point (bz_collision_term_static).

Callers that cannot allocate device memory -- code running inside another
framework's memory pool, under an allocator that forbids cudaMalloc, or a
plug-in restricted to the buffers it is handed -- call this entry point; it
keeps its scratch in the library's fixed-size static device arrays.  Its
output must equal that of bz_collision_term with the FP64 integrand (the
bar of the FP64 parity tests: bit for bit), and the oracle's, on two calls
in a row, the second taking the first call's masses as its previous masses,
in each mass mode; one call runs with the masses updated in place.  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _states(mask, nxc, np_, seeds):
    ns = bin(mask).count("1")
    return [I.encode(I.random_f(np_, ns, nxc, sd, 0.0, 0.5), mask) for sd in seeds]


CASES = [((1, 1, 1), (8, 8, 8), 0x7F, 32), ((2, 2, 1), (6, 6, 6), 0x13, 48)]


@pytest.mark.parametrize("mass_mode", [0, 1, 2])
@pytest.mark.parametrize("nx,np_,mask,N", CASES)
def test_static_entry_matches_collision_term_on_two_calls(nx, np_, mask, N, mass_mode):
    import torch
    from paper_1912_04457_gb300 import bz

    L, seed, dt, alpha = 2.0, 5, 0.01, 0.3
    nxc = int(np.prod(nx))
    st1, st2 = _states(mask, nxc, np_, (21, 22))
    s1, s2 = [torch.from_numpy(s.reshape(-1)).cuda() for s in (st1, st2)]
    fixed = np.random.default_rng(4).uniform(0.05, 0.4, size=(nxc, 4))

    # the existing entry point: two calls, the second using the first's masses for E
    h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=L, seed=seed, species_mask=mask, alpha_s=alpha, mass_mode=mass_mode)
    if mass_mode == bz.MASS_FIXED:
        h.set_masses(fixed)
    ref_A1 = torch.empty_like(s1)
    ref_A2 = torch.empty_like(s1)
    h.collision_term(s1, ref_A1, N, 0, dt, bz.PREC_F64)
    ref_m1 = h.get_masses()
    h.collision_term(s2, ref_A2, N, 1, dt, bz.PREC_F64)
    ref_m2 = h.get_masses()
    h.close()

    # the no-allocation entry point, two calls in a row on the same scratch
    m_in = torch.from_numpy(fixed.reshape(-1)).cuda() if mass_mode == bz.MASS_FIXED else None
    m1 = torch.empty(nxc * 4, dtype=torch.float64, device="cuda")
    m2 = torch.empty_like(m1)
    A1 = torch.empty_like(s1)
    A2 = torch.empty_like(s1)
    bz.collision_term_static(nx, 0.2, np_, L, seed, mask, alpha, mass_mode, s1, m_in, m1, A1, N, 0, dt)
    bz.collision_term_static(nx, 0.2, np_, L, seed, mask, alpha, mass_mode, s2, m1, m2, A2, N, 1, dt)
    torch.cuda.synchronize()

    assert np.array_equal(m1.cpu().numpy().reshape(nxc, 4), ref_m1)
    assert np.array_equal(m2.cpu().numpy().reshape(nxc, 4), ref_m2)
    assert np.array_equal(A1.cpu().numpy(), ref_A1.cpu().numpy())
    assert np.array_equal(A2.cpu().numpy(), ref_A2.cpu().numpy())
    assert int(A2.sum().item()) == 0 and int(A2.abs().sum().item()) > 0

    # and the oracle's, on the second call
    cfg = O.make_config(nx=nx, dx=0.2, np_=np_, L=L, seed=seed, species_mask=mask, alpha_s=alpha,
                        mass_mode=mass_mode)
    ref = O.collision(cfg, st2, ref_m2, N, step=1, dt=dt)["A"]
    assert np.array_equal(A2.cpu().numpy().reshape(ref.shape), ref)


def test_static_entry_with_masses_updated_in_place():
    """m2_in and m2_out the same buffer: the thermal masses of the second call
    are computed from the first call's, then overwrite them."""
    import torch
    from paper_1912_04457_gb300 import bz

    nx, np_, mask, N = (1, 1, 1), (8, 8, 8), 0x7F, 32
    L, seed, dt, alpha = 2.0, 5, 0.01, 0.3
    s1, s2 = [torch.from_numpy(s.reshape(-1)).cuda() for s in _states(mask, 1, np_, (31, 32))]
    h = bz.Handle(np_=np_, L=L, seed=seed, species_mask=mask, alpha_s=alpha)
    ref_A = torch.empty_like(s1)
    h.collision_term(s1, ref_A, N, 0, dt, bz.PREC_F64)
    h.collision_term(s2, ref_A, N, 1, dt, bz.PREC_F64)
    ref_m = h.get_masses()
    h.close()
    m = torch.empty(4, dtype=torch.float64, device="cuda")
    A = torch.empty_like(s1)
    bz.collision_term_static(nx, 0.2, np_, L, seed, mask, alpha, bz.MASS_THERMAL, s1, None, m, A, N, 0, dt)
    bz.collision_term_static(nx, 0.2, np_, L, seed, mask, alpha, bz.MASS_THERMAL, s2, m, m, A, N, 1, dt)
    torch.cuda.synchronize()
    assert np.array_equal(m.cpu().numpy().reshape(1, 4), ref_m)
    assert np.array_equal(A.cpu().numpy(), ref_A.cpu().numpy())


def test_static_entry_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1912_04457_gb300 import bz

    np_ = (48, 48, 48)          # 7 x 48^3 = 774144 cells > BZ_STATIC_MAX_CELLS
    ncell = 7 * 48 ** 3
    st = torch.zeros(ncell, dtype=torch.int64, device="cuda")
    A = torch.zeros_like(st)
    m2 = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(bz.BzError) as e:
        bz.collision_term_static((1, 1, 1), 1.0, np_, 3.0, 1, 0x7F, 0.3, bz.MASS_THERMAL, st, None,
                                 m2, A, 16)
    assert e.value.code == bz.BZ_EINVAL
    assert "static scratch" in str(e.value)
