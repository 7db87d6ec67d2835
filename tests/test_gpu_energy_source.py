"""bz_energy_source against the oracle, bit for bit: the integral
int N f / E (exact integer sum), the S_ex^0 part (1/2)((m^2 - m^2_prev)/dt) I
and the T_total term -(1/4) m^2 I of Eq. (current conservation), for
computed, massless and fixed masses, with and without previous masses."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,np_,mask,mass_mode,frange", [
    ((1, 1, 1), (8, 8, 8), 0x01, 0, (0.0, 0.6)),
    ((1, 1, 1), (6, 8, 10), 0x7F, 0, (0.0, 0.6)),
    ((2, 1, 3), (6, 6, 6), 0x13, 2, (-0.3, 0.6)),
    ((1, 1, 1), (8, 8, 8), 0x7F, 1, (0.0, 0.6)),
    ((1, 1, 1), (6, 6, 6), 0x01, 2, (-1e5, 1e5)),
])
def test_energy_source_bit_exact(nx, np_, mask, mass_mode, frange):
    import torch
    from paper_1912_04457_gb300 import bz
    nxc = nx[0] * nx[1] * nx[2]
    ns = bin(mask).count("1")
    h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=2.0, species_mask=mask, mass_mode=mass_mode)
    cfg = O.make_config(nx=nx, dx=0.2, np_=np_, L=2.0, species_mask=mask, mass_mode=mass_mode)
    st = I.encode(I.random_f(np_, ns, nxc, 17, *frange), mask)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    rng = np.random.default_rng(4)
    if mass_mode == 2:
        h.set_masses(rng.uniform(0.05, 0.5, size=(nxc, 4)))
    prev = rng.uniform(0.05, 0.5, size=(nxc, 4))
    dt = 0.013
    for m2_prev in (prev, None):
        out = h.energy_source(dev, dt, m2_prev).cpu().numpy().reshape(nxc, ns, 3)
        m2 = h.get_masses()
        ref = O.energy_source(cfg, st, m2, m2 if m2_prev is None else m2_prev, dt)
        assert np.array_equal(out, ref)
        if m2_prev is None or mass_mode == 1:
            assert np.all(out[..., 1] == 0.0)


def test_energy_source_argument_errors():
    import torch
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(np_=(6, 6, 6), species_mask=1, mass_mode=2)
    st = torch.zeros(216, dtype=torch.int64, device="cuda")
    with pytest.raises(bz.BzError):
        h.energy_source(st, 0.01)          # fixed masses never set
    h.set_masses(np.full((1, 4), 0.2))
    with pytest.raises(bz.BzError):
        h.energy_source(st, 0.0)           # dt must be positive
