"""Checkpoint / restart (bz_save, bz_load): the state, the step index and the
current thermal masses determine the rest of a run, so 2 + 2 steps through a
checkpoint equal 4 steps in one go, bit for bit; a checkpoint written for
another grid or species set, or a truncated file, is refused."""
import os

import numpy as np
import pytest

from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _handle(mask=0x13, seed=4):
    from paper_1912_04457_gb300 import bz
    return bz.Handle(nx=(4, 3, 1), dx=0.3, np_=(8, 8, 8), L=2.0, seed=seed, species_mask=mask, alpha_s=0.3)


def test_restart_is_bit_exact(tmp_path):
    import torch
    from paper_1912_04457_gb300 import bz
    mask, N, dt = 0x13, 40, 0.004
    st0 = I.encode(I.random_f((8, 8, 8), 3, 12, 8, 0.0, 0.5), mask).reshape(-1)
    h1 = _handle(mask)
    a = torch.from_numpy(st0.copy()).cuda()
    h1.step(a, dt, 4, N, bz.PREC_F32, step0=0)
    h2 = _handle(mask)
    b = torch.from_numpy(st0.copy()).cuda()
    h2.step(b, dt, 2, N, bz.PREC_F32, step0=0)
    path = str(tmp_path / "run.bzck")
    h2.save(b, 2, path)
    h3 = _handle(mask)
    c = torch.zeros_like(b)
    step = h3.load(c, path)
    assert step == 2 and torch.equal(c, b)
    assert np.array_equal(h3.get_masses(), h2.get_masses())
    h3.step(c, dt, 2, N, bz.PREC_F32, step0=step)
    assert torch.equal(c, a)
    assert int(c.sum().item()) == int(st0.sum())


def test_mismatched_or_truncated_checkpoint_is_refused(tmp_path):
    import torch
    from paper_1912_04457_gb300 import bz
    h = _handle(0x13)
    st = torch.from_numpy(I.encode(I.random_f((8, 8, 8), 3, 12, 9, 0.0, 0.5), 0x13).reshape(-1)).cuda()
    path = str(tmp_path / "a.bzck")
    h.save(st, 7, path)
    other = _handle(0x13, seed=5)          # another seed: another sample stream
    with pytest.raises(bz.BzError):
        other.load(torch.zeros_like(st), path)
    with open(path, "rb") as f:
        data = f.read()
    short = str(tmp_path / "short.bzck")
    with open(short, "wb") as f:
        f.write(data[: len(data) // 2])
    with pytest.raises(bz.BzError):
        h.load(torch.zeros_like(st), short)
    with pytest.raises(bz.BzError):
        h.load(torch.zeros_like(st), os.path.join(str(tmp_path), "missing.bzck"))
