"""Bounds-checked build (BZ_CHECK=1): the library is rebuilt with every
computed index of the collision and drift kernels tested before
its access, and small cases of each path run through it in a child process.
No index may fall outside its buffer, and the results stay those of the
default build: bit-identical to the oracle on the FP64 path and the drift,
within the FP32 tolerance on the FP32 path (its float-float re-evaluation
included), whose two work schedules (counter, one unit per warp) give the
same bits."""
import json
import os
import subprocess
import sys

import pytest

from paper_1912_04457_gb300 import bz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import oracle as O
from paper_1912_04457_gb300 import build as B, bz, inputs as I

bz.load(B.build(force=True, out_dir=sys.argv[2], extra=["-DBZ_CHECK=1"]))
assert bz.check_counts(reset=True) == (0, -1)
out = {}

def state(mask, nxc, np_, seed, lo=0.05, hi=0.5):
    return I.encode(I.random_f(np_, bin(mask).count("1"), nxc, seed, lo, hi), mask)

def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))

# collision, 7 species on a ragged grid: FP64 bit for bit, FP32 within tolerance
np_, mask = (6, 4, 8), 0x7F
h = bz.Handle(np_=np_, L=2.0, seed=5, species_mask=mask, alpha_s=0.3)
cfg = O.make_config(np_=np_, L=2.0, seed=5, species_mask=mask, alpha_s=0.3)
st = state(mask, 1, np_, 21)
m2 = O.masses(cfg, st)
A = torch.empty(st.size, dtype=torch.int64, device="cuda")
h.collision_term(torch.from_numpy(st.reshape(-1)).cuda(), A, 32, 3, 0.01, bz.PREC_F64)
ref = O.collision(cfg, st, m2, 32, step=3, dt=0.01)["A"]
out["f64_equal"] = bool(np.array_equal(A.cpu().numpy().reshape(ref.shape), ref))
h.reset_masses()
h.collision_term(torch.from_numpy(st.reshape(-1)).cuda(), A, 32, 3, 0.01, bz.PREC_F32)
ref23 = O.collision(cfg, st, m2, 32, step=3, dt=0.01, ubits=23)["A"]
out["f32_rel_l2"] = rel_l2(A.cpu().numpy().reshape(ref23.shape), ref23)
# the same through the counter schedule (warps take units from a global counter)
import os
os.environ["BZ_F32_SCHEDULE"] = "counter"
A2 = torch.empty_like(A)
h.reset_masses()
h.collision_term(torch.from_numpy(st.reshape(-1)).cuda(), A2, 32, 3, 0.01, bz.PREC_F32)
del os.environ["BZ_F32_SCHEDULE"]
out["f32_counter_equal"] = bool(torch.equal(A, A2))

# streaming drift with the force term on an inhomogeneous grid, several species
nx, np_, mask = (3, 2, 4), (4, 6, 4), 0x03
nxc = 24
h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=2.0, seed=1, species_mask=mask, alpha_s=0.3, mass_mode=2)
cfg = O.make_config(nx=nx, dx=0.2, np_=np_, L=2.0, seed=1, species_mask=mask, alpha_s=0.3, mass_mode=2)
cfg.force = 1
h.set_force_term(True)
m2 = np.random.default_rng(3).uniform(0.0, 0.5, size=(nxc, 4))
h.set_masses(m2)
st = state(mask, nxc, np_, 8, -0.2, 0.6)
dst = torch.empty(st.size, dtype=torch.int64, device="cuda")
h.drift(torch.from_numpy(st.reshape(-1)).cuda(), dst, 0.05)
ref = O.drift(cfg, st, m2, 0.05).reshape(-1)
out["drift_equal"] = bool(np.array_equal(dst.cpu().numpy(), ref))

# the row kernel (n_z above the streaming kernel's buffer), with the force term
nx, np_, mask = (2, 2, 41), (4, 4, 4), 0x01
nxc = 164
h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=2.0, seed=1, species_mask=mask, alpha_s=0.3, mass_mode=2)
cfg = O.make_config(nx=nx, dx=0.2, np_=np_, L=2.0, seed=1, species_mask=mask, alpha_s=0.3, mass_mode=2)
cfg.force = 1
h.set_force_term(True)
m2 = np.random.default_rng(4).uniform(0.0, 0.5, size=(nxc, 4))
h.set_masses(m2)
st = state(mask, nxc, np_, 9, 0.0, 0.6)
dst = torch.empty(st.size, dtype=torch.int64, device="cuda")
h.drift(torch.from_numpy(st.reshape(-1)).cuda(), dst, 0.05)
out["row_drift_equal"] = bool(np.array_equal(dst.cpu().numpy(), O.drift(cfg, st, m2, 0.05).reshape(-1)))

torch.cuda.synchronize()
out["count"], out["first_bad"] = bz.check_counts()
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_checked_build_finds_no_index_outside_its_buffer(tmp_path):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "checked")], capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["count"] == 0 and res["first_bad"] == -1, res
    assert res["f64_equal"] and res["drift_equal"] and res["row_drift_equal"], res
    assert res["f32_rel_l2"] <= 2e-5 and res["f32_counter_equal"], res


def test_default_build_has_no_checks():
    # the default build compiles the checks away and says so (no GPU needed)
    with pytest.raises(bz.BzError) as e:
        bz.check_counts()
    assert e.value.code == bz.BZ_EINVAL
