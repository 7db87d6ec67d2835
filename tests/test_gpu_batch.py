"""Batched ensemble (bz_batch_*): every box of one persistent, graph-replayed
launch equals the same box stepped alone through a handle with the FP32
integrand, bit for bit (same kernels on the same Philox counters, integer
deposits); number is conserved per box; the autotuner picks a valid shape."""
import numpy as np
import pytest

from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _small_batch():
    specs = [((6, 6, 6), 0x01, 40, 0.30, 0), ((8, 8, 8), 0x7F, 64, 0.25, 0), ((10, 10, 10), 0x01, 33, 0.35, 1),
             ((6, 8, 10), 0x7F, 96, 0.20, 0), ((12, 12, 12), 0x01, 128, 0.40, 0), ((4, 6, 8), 0x13, 50, 0.30, 0)]
    boxes, states = [], []
    for i, (np_, mask, N, a, mm) in enumerate(specs):
        boxes.append({"np_": np_, "L": 2.0, "species_mask": mask, "nsamples": N, "alpha_s": a,
                      "mass_mode": mm, "box_id": 7 + i, "seed": 11})
        states.append(I.encode(I.random_f(np_, bin(mask).count("1"), 1, 30 + i, 0.0, 0.5), mask))
    return boxes, states


def test_batch_matches_single_boxes_bit_for_bit():
    import torch
    from paper_1912_04457_gb300 import bz
    boxes, states = _small_batch()
    dt, nsteps = 0.01, 3
    B = bz.Batch(boxes)
    flat = torch.from_numpy(np.concatenate([s.reshape(-1) for s in states])).cuda()
    assert flat.numel() == B.ncell
    mom = torch.empty(nsteps * B.nslots_total * 5, dtype=torch.float64, device="cuda")
    B.step(flat, dt, nsteps, step0=4, moments_out=mom)
    torch.cuda.synchronize()
    got = flat.cpu().numpy()
    gmom = mom.cpu().numpy().reshape(nsteps, B.nslots_total, 5)
    tun = B.tuning()
    assert tun["chunk"] >= 1 and tun["blocks_per_sm"] in (4, 5, 6)
    m_batch = B.get_masses()
    for i, (bx, st) in enumerate(zip(boxes, states)):
        h = bz.Handle(np_=bx["np_"], L=bx["L"], seed=bx["seed"], box=bx["box_id"],
                      species_mask=bx["species_mask"], alpha_s=bx["alpha_s"], mass_mode=bx["mass_mode"])
        dev = torch.from_numpy(st.reshape(-1)).cuda()
        hm = torch.empty(nsteps * h.nslots * 5, dtype=torch.float64, device="cuda")
        h.step(dev, dt, nsteps, bx["nsamples"], bz.PREC_F32, step0=4, moments_out=hm)
        lo, hi = B.cell_offsets[i], B.cell_offsets[i + 1]
        ref = dev.cpu().numpy()
        assert np.array_equal(got[lo:hi], ref), "box %d state" % i
        assert int(ref.sum()) == int(st.sum())
        s0, s1 = B.slot_offsets[i], B.slot_offsets[i + 1]
        assert np.array_equal(gmom[:, s0:s1, :], hm.cpu().numpy().reshape(nsteps, h.nslots, 5)), "box %d moments" % i
        assert np.array_equal(m_batch[i], h.get_masses()[0]), "box %d masses" % i
        h.close()
    # a second call continues from the previous masses and the given step index
    B.step(flat, dt, 1, step0=7)
    torch.cuda.synchronize()
    assert int(flat.sum().item()) == int(sum(int(s.sum()) for s in states))
    B.close()


def test_batch_rejects_bad_boxes():
    from paper_1912_04457_gb300 import bz
    with pytest.raises(bz.BzError):
        bz.Batch([{"np_": (4, 4, 4), "L": 2.0, "species_mask": 0, "nsamples": 8, "alpha_s": 0.3}])
    with pytest.raises(bz.BzError):
        bz.Batch([{"np_": (4, 4, 4), "L": 2.0, "species_mask": 1, "nsamples": 8, "alpha_s": 0.3,
                   "mass_mode": 2}])
