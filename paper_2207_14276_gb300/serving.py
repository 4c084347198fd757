"""Python binding of the continuous-batching server (argument marshalling only).

The server, its queue, lanes, streams and batching policy are native (see the
nnp_server_* entry points in include/nnp.h); this wrapper keeps the host
buffers of in-flight requests alive until they are polled.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check, lib


class Server:
    def __init__(self, potential, n_lanes=2, max_batch_atoms=65536, max_batch_systems=256):
        self.potential = potential          # keeps the model handle alive
        h = ctypes.c_void_p()
        check(lib().nnp_server_create(potential._h, n_lanes, int(max_batch_atoms),
                                      int(max_batch_systems), ctypes.byref(h)))
        self._s = h
        self._inflight = {}

    def close(self):
        if getattr(self, "_s", None):
            lib().nnp_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, coords, species, box=None, mask=None):
        x = np.ascontiguousarray(coords, dtype=np.float32)
        sp = np.ascontiguousarray(species, dtype=np.uint8)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        b = None if box is None else (ctypes.c_double * 3)(*[float(v) for v in box])
        rid = ctypes.c_int()
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        check(lib().nnp_server_register(self._s, x.shape[0], vp(x), vp(sp), vp(m), b,
                                        ctypes.byref(rid)))
        return rid.value

    def submit(self, coords, species=None, box=None, mask=None, resident_id=-1):
        """Queue one request; returns a ticket.  For resident_id >= 0, coords are the
        new coordinates of the resident system's first len(coords) atoms."""
        x = np.ascontiguousarray(coords, dtype=np.float32)
        n = x.shape[0]
        keep = [x]
        r = _lib.RequestT()
        r.n_atoms = n
        r.coords = x.ctypes.data
        r.resident_id = resident_id
        if resident_id < 0:
            sp = np.ascontiguousarray(species, dtype=np.uint8)
            keep.append(sp)
            r.species = sp.ctypes.data
            if mask is not None:
                m = np.ascontiguousarray(mask, dtype=np.uint8)
                keep.append(m)
                r.mask = m.ctypes.data
            if box is not None:
                r.periodic = 1
                for c in range(3):
                    r.box[c] = float(box[c])
        E = np.zeros(1, dtype=np.float64)
        F = np.zeros((n, 3), dtype=np.float32)
        r.energy = E.ctypes.data
        r.forces = F.ctypes.data
        t = ctypes.c_uint64()
        check(lib().nnp_server_submit(self._s, ctypes.byref(r), ctypes.byref(t)))
        self._inflight[t.value] = (E, F, keep)
        return t.value

    def poll(self, ticket, wait=True):
        """(status, energy, forces, latency_s) once done; None while pending."""
        lat = ctypes.c_double()
        rc = lib().nnp_server_poll(self._s, ticket, 1 if wait else 0, ctypes.byref(lat))
        if rc == _lib.NNP_PENDING:
            return None
        E, F, _ = self._inflight.pop(ticket)
        return rc, float(E[0]), F, lat.value

    def stats(self):
        b, r = ctypes.c_longlong(), ctypes.c_longlong()
        check(lib().nnp_server_stats(self._s, ctypes.byref(b), ctypes.byref(r)))
        return b.value, r.value
