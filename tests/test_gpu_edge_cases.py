"""Edge cases of the collision term through the C ABI: an empty (all-zero)
state, the maximum sample count per anchor, the maximum momentum cells along
one axis, and argument errors at the limits."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _pair(np_, mask, seed=3, mass_mode=0):
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(np_=np_, L=2.0, seed=seed, species_mask=mask, mass_mode=mass_mode)
    cfg = O.make_config(np_=np_, L=2.0, seed=seed, species_mask=mask, mass_mode=mass_mode)
    return h, cfg


@pytest.mark.parametrize("prec", [0, 1])
def test_empty_state_gives_nothing(prec):
    import torch
    h, _ = _pair((6, 6, 6), 0x7F)
    st = torch.zeros(7 * 216, dtype=torch.int64, device="cuda")
    A = torch.full_like(st, 123)
    h.collision_term(st, A, 64, 0, 0.01, prec)
    assert int(A.abs().sum().item()) == 0
    assert np.all(h.get_masses() == 0.0)
    assert np.all(h.flags() == 0)


def test_maximum_samples_per_anchor():
    """N = 2^20 (the limit) on a 4^3 gluon box: the FP32 path within 2e-5 of
    the oracle on the same 23-bit uniforms, exact conservation."""
    import torch
    from paper_1912_04457_gb300 import bz
    np_, N = (4, 4, 4), 1 << 20
    h, cfg = _pair(np_, 0x01, seed=8)
    st = I.encode(I.random_f(np_, 1, 1, 4, 0.05, 0.6), 0x01)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(torch.from_numpy(st.reshape(-1)).cuda(), A, N, 1, 0.01, bz.PREC_F32)
    ref = O.collision(cfg, st, O.masses(cfg, st), N, step=1, dt=0.01, ubits=23)["A"].reshape(-1)
    got = A.cpu().numpy()
    assert int(got.sum()) == 0
    assert np.linalg.norm((got - ref).astype(float)) / np.linalg.norm(ref.astype(float)) <= 2e-5


def test_maximum_cells_along_one_axis():
    """256 momentum cells along x (the limit), 7 species: FP64 bit-identical."""
    import torch
    from paper_1912_04457_gb300 import bz
    np_ = (256, 2, 4)
    h, cfg = _pair(np_, 0x7F, seed=9)
    st = I.encode(I.random_f(np_, 7, 1, 6, 0.0, 0.5), 0x7F)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(torch.from_numpy(st.reshape(-1)).cuda(), A, 8, 2, 0.01, bz.PREC_F64)
    ref = O.collision(cfg, st, O.masses(cfg, st), 8, step=2, dt=0.01)["A"].reshape(-1)
    assert np.array_equal(A.cpu().numpy(), ref)


def test_state_warnings_count_negative_and_pauli_cells():
    """bz_moments counts cells with f < 0 and (anti)quark cells with f > 1."""
    import torch
    from paper_1912_04457_gb300 import bz
    np_, mask = (6, 6, 6), 0x13          # g, u, ubar
    h, _ = _pair(np_, mask)
    f = I.random_f(np_, 3, 1, 12, 0.0, 0.9)
    f[0, 0, :5] = -0.01                  # 5 negative gluon cells
    f[1, 0, 10:17] = 1.2                 # 7 quark cells above 1
    f[2, 0, 3] = -0.5                    # 1 negative antiquark cell
    f[2, 0, 4] = 1.0 + 1e-9              # 1 antiquark cell just above 1
    f[0, 0, 20] = 3.0                    # gluons may exceed 1
    st = torch.from_numpy(I.encode(f, mask).reshape(-1)).cuda()
    mom = torch.empty(3 * 5, dtype=torch.float64, device="cuda")
    h.clear_flags()
    h.moments(st, mom)
    assert list(h.state_flags()) == [6, 8]
    h.clear_flags()
    assert list(h.state_flags()) == [0, 0]


def test_limits_are_refused():
    import torch
    from paper_1912_04457_gb300 import bz
    h, _ = _pair((4, 4, 4), 0x01)
    st = torch.zeros(64, dtype=torch.int64, device="cuda")
    A = torch.empty_like(st)
    for N in (0, (1 << 20) + 1):
        with pytest.raises(bz.BzError):
            h.collision_term(st, A, N, 0, 0.01, bz.PREC_F32)
    with pytest.raises(bz.BzError):
        bz.Handle(np_=(3, 5, 7), L=2.0)            # a cell centred at p = 0
    with pytest.raises(bz.BzError):
        bz.Handle(np_=(257, 2, 2), L=2.0)          # beyond 256 cells per axis
