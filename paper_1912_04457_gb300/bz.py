"""Thin ctypes binding of libbz (include/bz.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module checks the
tensors (device, dtype, shape, contiguity), passes their data pointers and
the current torch stream, and turns negative return codes into exceptions.
There is no fallback: if libbz.so is missing, `load()` raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbz.so")

BZ_OK, BZ_EINVAL, BZ_ENOMEM, BZ_ECUDA, BZ_EOVERFLOW, BZ_ENODEV = 0, -1, -2, -3, -4, -5
PREC_F64, PREC_F32 = 0, 1
SAMPLER_SYMMETRIC, SAMPLER_PLAIN = 0, 1
SAMPLER_LEARNED = 2
MASS_THERMAL, MASS_MASSLESS, MASS_FIXED = 0, 1, 2
RECORD_BYTES = 32  # struct { int64 anchor; float w; float y[5]; }
KERNELS = ("masses", "drift", "collide", "fixup", "moments", "convert")


class BzGrid(C.Structure):
    _fields_ = [("nx", C.c_int32 * 3), ("dx", C.c_double), ("np", C.c_int32 * 3), ("L", C.c_double),
                ("seed", C.c_uint64), ("box", C.c_uint32), ("reserved", C.c_uint32)]


class BzBox(C.Structure):
    _fields_ = [("np", C.c_int32 * 3), ("L", C.c_double), ("species_mask", C.c_uint32),
                ("nsamples", C.c_int32), ("alpha_s", C.c_double), ("mass_mode", C.c_int32),
                ("box_id", C.c_uint32), ("seed", C.c_uint64)]


class BzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libbz error %d: %s" % (code, msg))
        self.code = code


_lib = None

# name -> (restype, argtypes)
_P, _I32, _I64, _D, _U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint32
SIGNATURES = {
    "bz_init_grid": (C.c_int, [C.POINTER(_P), C.POINTER(BzGrid)]),
    "bz_destroy": (C.c_int, [_P]),
    "bz_last_error": (C.c_char_p, [_P]),
    "bz_set_species": (C.c_int, [_P, _U32, _D, C.c_int]),
    "bz_query_sizes": (C.c_int, [_P, _P, _P, _P]),
    "bz_collision_term": (C.c_int, [_P, _P, _P, _I32, _I32, _D, _I32, _I32, _P]),
    "bz_drift": (C.c_int, [_P, _P, _P, _D, _P]),
    "bz_step": (C.c_int, [_P, _P, _D, _I32, _I32, _I32, _I32, _P, _P]),
    "bz_moments": (C.c_int, [_P, _P, _P, _P]),
    "bz_get_masses": (C.c_int, [_P, _P]),
    "bz_set_masses": (C.c_int, [_P, _P]),
    "bz_reset_masses": (C.c_int, [_P]),
    "bz_get_flags": (C.c_int, [_P, _P]),
    "bz_clear_flags": (C.c_int, [_P]),
    "bz_set_anchor_subset": (C.c_int, [_P, _I64, _I64]),
    "bz_get_state_flags": (C.c_int, [_P, _P]),
    "bz_set_uniform_bits": (C.c_int, [_P, _I32]),
    "bz_set_force_term": (C.c_int, [_P, _I32]),
    "bz_set_parameterisation": (C.c_int, [_P, _I32]),
    "bz_set_matrix_element": (C.c_int, [_P, _I32, _I32, _P, _P]),
    "bz_energy_source": (C.c_int, [_P, _P, _P, C.c_double, _P, _P]),
    "bz_set_equilibrium": (C.c_int, [_P, C.c_int, _D, _P]),
    "bz_profile": (C.c_int, [_P, C.c_int]),
    "bz_profile_read": (C.c_int, [_P, _P, _P, _I32]),
    "bz_collision_term_static": (C.c_int, [C.POINTER(BzGrid), _U32, _D, _I32, _P, _P, _P, _P, _I32,
                                           _I32, _D, _P, C.c_char_p, _I32]),
    "bz_batch_create": (C.c_int, [C.POINTER(_P), _I32, _P]),
    "bz_batch_destroy": (C.c_int, [_P]),
    "bz_batch_last_error": (C.c_char_p, [_P]),
    "bz_batch_layout": (C.c_int, [_P, _P, _P]),
    "bz_batch_step": (C.c_int, [_P, _P, _D, _I32, _I32, _P, _P]),
    "bz_batch_tuning": (C.c_int, [_P, _P, _P, _P]),
    "bz_batch_get_masses": (C.c_int, [_P, _P]),
    "bz_batch_get_flags": (C.c_int, [_P, _P]),
    "bz_collision_audit": (C.c_int, [_P, _P, _P, _I32, _I32, _D, _I32, _P, _P]),
    "bz_save": (C.c_int, [_P, _P, _I64, C.c_char_p]),
    "bz_load": (C.c_int, [_P, _P, _P, C.c_char_p]),
    "bz_proposal_nparams": (C.c_int, []),
    "bz_proposal_init": (C.c_int, [_P, C.c_uint64]),
    "bz_proposal_get_params": (C.c_int, [_P, _P]),
    "bz_proposal_set_params": (C.c_int, [_P, _P]),
    "bz_record": (C.c_int, [_P, _P, _I32, _I32, _D, _I32, _P, _I64, _P, _P]),
    "bz_proposal_grad": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "bz_proposal_train": (C.c_int, [_P, _P, _I64, _I32, _I32, _D, _P, _P]),
    "bz_proposal_infer": (C.c_int, [_P, _P]),
    "bz_proposal_anchor_params": (C.c_int, [_P, _P, _P]),
    "bz_set_step_sampler": (C.c_int, [_P, _I32]),
    "bz_version": (C.c_char_p, []),
    "bz_check_counts": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32]),
}


def load(path=LIB_PATH):
    """Loads libbz.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libbz.so not found at %s; run __graft_entry__.build() first" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return C.c_void_p(t.data_ptr())


class Handle:
    """One phase-space grid on the current CUDA device (bz_init_grid)."""

    def __init__(self, nx=(1, 1, 1), dx=1.0, np_=(20, 20, 20), L=2.0, seed=1, box=0,
                 species_mask=1, alpha_s=0.3, mass_mode=MASS_THERMAL):
        self.lib = load()
        g = BzGrid()
        g.nx[:] = list(nx)
        g.dx = dx
        g.np[:] = list(np_)
        g.L = L
        g.seed = seed
        g.box = box
        h = C.c_void_p()
        rc = self.lib.bz_init_grid(C.byref(h), C.byref(g))
        if rc != BZ_OK:
            raise BzError(rc, self.lib.bz_last_error(None).decode())
        self.h = h
        self.nx, self.np_ = tuple(nx), tuple(np_)
        self.set_species(species_mask, alpha_s, mass_mode)

    def _check(self, rc):
        if rc != BZ_OK:
            raise BzError(rc, self.lib.bz_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.bz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ----------------------------------------------------
    def set_species(self, species_mask, alpha_s=0.3, mass_mode=MASS_THERMAL):
        self._check(self.lib.bz_set_species(self.h, species_mask, alpha_s, mass_mode))
        ns, nx, npc = C.c_int32(), C.c_int64(), C.c_int64()
        self._check(self.lib.bz_query_sizes(self.h, C.byref(ns), C.byref(nx), C.byref(npc)))
        self.nslots, self.nxc, self.npc = ns.value, nx.value, npc.value
        self.ncell = self.nslots * self.nxc * self.npc

    @property
    def shape(self):
        return (self.nslots, self.nxc, self.npc)

    def set_uniform_bits(self, bits):
        self._check(self.lib.bz_set_uniform_bits(self.h, bits))

    def set_matrix_element(self, row, terms):
        """terms: [(coef, (a, b, c, d, e, f)), ...] (empty: default row)."""
        coef = np.ascontiguousarray([c for c, _ in terms], dtype=np.float64)
        exps = np.ascontiguousarray([e for _, e in terms], dtype=np.int32).reshape(-1)
        self._check(self.lib.bz_set_matrix_element(self.h, row, len(terms),
                                                   coef.ctypes.data_as(C.c_void_p) if len(terms) else None,
                                                   exps.ctypes.data_as(C.c_void_p) if len(terms) else None))

    def set_parameterisation(self, which):
        """0: k2 eliminated (default), 1: k3 eliminated (FP64 path, uniform samples)."""
        self._check(self.lib.bz_set_parameterisation(self.h, which))

    def set_force_term(self, enable=True):
        self._check(self.lib.bz_set_force_term(self.h, 1 if enable else 0))

    def set_anchor_subset(self, stride=1, offset=0):
        self._check(self.lib.bz_set_anchor_subset(self.h, stride, offset))

    def set_equilibrium(self, enable, T=0.5, mu=None):
        mu = np.ascontiguousarray(mu if mu is not None else np.zeros(7), dtype=np.float64)
        self._check(self.lib.bz_set_equilibrium(self.h, 1 if enable else 0, T,
                                                mu.ctypes.data_as(C.c_void_p)))

    def get_masses(self):
        out = np.zeros((self.nxc, 4))
        self._check(self.lib.bz_get_masses(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_masses(self, m2):
        m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(self.nxc, 4)
        self._check(self.lib.bz_set_masses(self.h, m2.ctypes.data_as(C.c_void_p)))

    def reset_masses(self):
        self._check(self.lib.bz_reset_masses(self.h))

    def flags(self):
        out = np.zeros(4, dtype=np.int64)
        self._check(self.lib.bz_get_flags(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def state_flags(self):
        """[cells with f < 0, fermion cells with f > 1] counted by the moments evaluations."""
        out = np.zeros(2, dtype=np.int64)
        self._check(self.lib.bz_get_state_flags(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def clear_flags(self):
        self._check(self.lib.bz_clear_flags(self.h))

    def profile(self, enable=True):
        self._check(self.lib.bz_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel: (ms summed, launches)} of this handle's launches while profiling."""
        n = len(KERNELS)
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        self._check(self.lib.bz_profile_read(self.h, ms.ctypes.data_as(C.c_void_p),
                                             cnt.ctypes.data_as(C.c_void_p), n))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}

    # -- learned proposal ----------------------------------------------------
    def proposal_init(self, seed=1):
        self._check(self.lib.bz_proposal_init(self.h, seed))

    def proposal_params(self):
        out = np.zeros(self.lib.bz_proposal_nparams(), dtype=np.float32)
        self._check(self.lib.bz_proposal_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_proposal_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.lib.bz_proposal_nparams()
        self._check(self.lib.bz_proposal_set_params(self.h, p.ctypes.data_as(C.c_void_p)))

    def record(self, state, nsamples, step=0, dt=0.01, unit_stride=1, max_records=1 << 20, stream=None):
        """Uniform-sampler records (uint8 CUDA tensor of max_records x 32 bytes), count."""
        import torch
        rec = torch.empty(max_records * RECORD_BYTES, dtype=torch.uint8, device="cuda")
        n = C.c_int64()
        self._check(self.lib.bz_record(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), nsamples,
                                       step, dt, unit_stride, C.c_void_p(rec.data_ptr()), max_records,
                                       C.byref(n), _stream_ptr(stream)))
        return rec, n.value

    def proposal_grad(self, records, n, stream=None):
        import torch
        npar = self.lib.bz_proposal_nparams()
        grad = torch.empty(npar, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self.lib.bz_proposal_grad(self.h, C.c_void_p(records.data_ptr()), n,
                                              C.c_void_p(grad.data_ptr()), C.c_void_p(loss.data_ptr()),
                                              _stream_ptr(stream)))
        return grad, loss

    def proposal_train(self, records, n, steps, batch=16384, lr=1e-3, stream=None):
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(self.lib.bz_proposal_train(self.h, C.c_void_p(records.data_ptr()), n, steps, batch, lr,
                                               losses.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return losses[:steps]

    def proposal_infer(self, stream=None):
        self._check(self.lib.bz_proposal_infer(self.h, _stream_ptr(stream)))

    def anchor_params(self):
        out = np.zeros((self.ncell, 8), dtype=np.float32)
        self._check(self.lib.bz_proposal_anchor_params(self.h, out.ctypes.data_as(C.c_void_p), None))
        return out

    def set_anchor_params(self, prm):
        prm = np.ascontiguousarray(prm, dtype=np.float32).reshape(self.ncell, 8)
        self._check(self.lib.bz_proposal_anchor_params(self.h, None, prm.ctypes.data_as(C.c_void_p)))

    def set_step_sampler(self, sampler):
        self._check(self.lib.bz_set_step_sampler(self.h, sampler))

    # -- the hot path -------------------------------------------------------
    def collision_term(self, state, A, nsamples, step=0, dt=0.01, prec=PREC_F64,
                       sampler=SAMPLER_SYMMETRIC, stream=None):
        import torch
        self._check(self.lib.bz_collision_term(
            self.h, _dev_ptr(state, torch.int64, self.ncell, "state"),
            _dev_ptr(A, torch.int64, self.ncell, "A"), nsamples, step, dt, prec, sampler,
            _stream_ptr(stream)))

    def collision_audit(self, state, A, nsamples, step=0, dt=0.01, sampler=SAMPLER_SYMMETRIC, stream=None):
        """FP64 collision term into A plus the conservation audit (numpy float64 [8])."""
        import torch
        out = np.zeros(8, dtype=np.float64)
        self._check(self.lib.bz_collision_audit(
            self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), _dev_ptr(A, torch.int64, self.ncell, "A"),
            nsamples, step, dt, sampler, out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return out

    def save(self, state, step, path):
        """Checkpoint of state (CUDA int64 tensor), the step index and the current masses."""
        import torch
        self._check(self.lib.bz_save(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), step,
                                     os.fsencode(path)))

    def load(self, state, path):
        """Restores a checkpoint into state (CUDA int64 tensor); returns the saved step index."""
        import torch
        step = C.c_int64()
        self._check(self.lib.bz_load(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), C.byref(step),
                                     os.fsencode(path)))
        return step.value

    def drift(self, state_in, state_out, dt, stream=None):
        import torch
        self._check(self.lib.bz_drift(self.h, _dev_ptr(state_in, torch.int64, self.ncell, "in"),
                                      _dev_ptr(state_out, torch.int64, self.ncell, "out"), dt,
                                      _stream_ptr(stream)))

    def step(self, state, dt, nsteps, nsamples, prec=PREC_F32, step0=0, moments_out=None,
             stream=None):
        import torch
        mptr = None
        if moments_out is not None:
            mptr = _dev_ptr(moments_out, torch.float64, nsteps * self.nxc * self.nslots * 5,
                            "moments_out")
        self._check(self.lib.bz_step(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), dt,
                                     nsteps, nsamples, prec, step0, mptr, _stream_ptr(stream)))

    def moments(self, state, out, stream=None):
        import torch
        self._check(self.lib.bz_moments(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"),
                                        _dev_ptr(out, torch.float64, self.nxc * self.nslots * 5, "out"),
                                        _stream_ptr(stream)))

    def energy_source(self, state, dt, m2_prev=None, out=None, stream=None):
        """Per (x cell, slot): [int N f / E, S_ex^0 part, T_total term] (bz_energy_source);
        m2_prev: host [nx, 4] masses of the previous evaluation, or None."""
        import torch
        if out is None:
            out = torch.empty(self.nxc * self.nslots * 3, dtype=torch.float64, device=state.device)
        prev = None if m2_prev is None else np.ascontiguousarray(m2_prev, dtype=np.float64).reshape(self.nxc, 4)
        self._check(self.lib.bz_energy_source(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"),
                                              None if prev is None else prev.ctypes.data_as(C.c_void_p),
                                              C.c_double(dt),
                                              _dev_ptr(out, torch.float64, self.nxc * self.nslots * 3, "out"),
                                              _stream_ptr(stream)))
        return out


class Batch:
    """Independent homogeneous boxes stepped together (bz_batch_*).  `boxes`:
    list of dicts with np_, L, species_mask, nsamples, alpha_s, mass_mode,
    box_id, seed."""

    def __init__(self, boxes):
        self.lib = load()
        arr = (BzBox * len(boxes))()
        for i, b in enumerate(boxes):
            arr[i].np[:] = list(b["np_"])
            arr[i].L = b["L"]
            arr[i].species_mask = b["species_mask"]
            arr[i].nsamples = b["nsamples"]
            arr[i].alpha_s = b["alpha_s"]
            arr[i].mass_mode = b.get("mass_mode", MASS_THERMAL)
            arr[i].box_id = b.get("box_id", i)
            arr[i].seed = b.get("seed", 1)
        h = C.c_void_p()
        rc = self.lib.bz_batch_create(C.byref(h), len(boxes), C.cast(arr, C.c_void_p))
        if rc != BZ_OK:
            raise BzError(rc, self.lib.bz_batch_last_error(None).decode())
        self.h = h
        self.nboxes = len(boxes)
        self.cell_offsets = np.zeros(self.nboxes + 1, dtype=np.int64)
        self.slot_offsets = np.zeros(self.nboxes + 1, dtype=np.int32)
        self._check(self.lib.bz_batch_layout(self.h, self.cell_offsets.ctypes.data_as(C.c_void_p),
                                             self.slot_offsets.ctypes.data_as(C.c_void_p)))
        self.ncell = int(self.cell_offsets[-1])
        self.nslots_total = int(self.slot_offsets[-1])

    def _check(self, rc):
        if rc != BZ_OK:
            raise BzError(rc, self.lib.bz_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.bz_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, state, dt, nsteps, step0=0, moments_out=None, stream=None):
        import torch
        mptr = None
        if moments_out is not None:
            mptr = _dev_ptr(moments_out, torch.float64, nsteps * self.nslots_total * 5, "moments_out")
        self._check(self.lib.bz_batch_step(self.h, _dev_ptr(state, torch.int64, self.ncell, "state"), dt,
                                           nsteps, step0, mptr, _stream_ptr(stream)))

    def tuning(self):
        ch, bps, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._check(self.lib.bz_batch_tuning(self.h, C.byref(ch), C.byref(bps), C.byref(ms)))
        return {"chunk": ch.value, "blocks_per_sm": bps.value, "collide_ms": ms.value}

    def get_masses(self):
        out = np.zeros((self.nboxes, 4))
        self._check(self.lib.bz_batch_get_masses(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def flags(self):
        out = np.zeros(4, dtype=np.int64)
        self._check(self.lib.bz_batch_get_flags(self.h, out.ctypes.data_as(C.c_void_p)))
        return out


def collision_term_static(nx, dx, np_, L, seed, species_mask, alpha_s, mass_mode, state, m2_in,
                          m2_out, A, nsamples, step=0, dt=0.01, box=0, stream=None):
    """bz_collision_term_static: the FP64 collision increment with no device
    allocation (scratch in the library's static device arrays)."""
    import torch
    lib = load()
    g = BzGrid()
    g.nx[:] = list(nx)
    g.dx = dx
    g.np[:] = list(np_)
    g.L = L
    g.seed = seed
    g.box = box
    nxc = int(np.prod(nx))
    ncell = bin(species_mask).count("1") * nxc * int(np.prod(np_))
    m2p = None if m2_in is None else _dev_ptr(m2_in, torch.float64, nxc * 4, "m2_in")
    buf = C.create_string_buffer(512)
    rc = lib.bz_collision_term_static(C.byref(g), species_mask, alpha_s, mass_mode,
                                      _dev_ptr(state, torch.int64, ncell, "state"), m2p,
                                      _dev_ptr(m2_out, torch.float64, nxc * 4, "m2_out"),
                                      _dev_ptr(A, torch.int64, ncell, "A"), nsamples, step, dt,
                                      _stream_ptr(stream), buf, 512)
    if rc != BZ_OK:
        raise BzError(rc, buf.value.decode())


def version():
    return load().bz_version().decode()


def check_counts(reset=False):
    """(indices outside their buffers, one of them or -1) of a library built
    with BZ_CHECK=1; raises BzError in the default build."""
    lib = load()
    n, first = C.c_int64(), C.c_int64()
    rc = lib.bz_check_counts(C.byref(n), C.byref(first), 1 if reset else 0)
    if rc != 0:
        raise BzError(rc, lib.bz_last_error(None).decode())
    return n.value, first.value
