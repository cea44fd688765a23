"""Process-parallel execution of the oracle's local solves.

TEST INFRASTRUCTURE ONLY, like the rest of :mod:`oracle`: it serves the CPU
baseline's all-cores mode and the tests, never the GPU library.

The same arithmetic as :class:`oracle.Sweeper`; only the place where the local
solves run changes.  Subdomain ``i`` belongs to worker ``position(i) mod P``
(one process per worker, started with ``spawn``), which builds its own
:class:`oracle.Decomposition` and the sparse LU factors of its subdomains only,
the analogue of the paper's distribution of the subdomains over MPI ranks
(Section 6).  The independent local solves of one stage (the subdomains of one
anti-diagonal in a sweep step, every subdomain in ``S``, the liftings and the
reconstructions) go to their owners at once; only interface data and subdomain
vectors cross processes.  Every worker factors the same matrices and runs the
same solves as the serial sweeper, so the results are equal bit for bit.
"""
import multiprocessing as mp

import numpy as np

from .decomposition import Decomposition
from .sweeping import Sweeper

_DEC = None          # this worker's Decomposition


def _init(args, kwargs):
    global _DEC
    _DEC = Decomposition(*args, **kwargs)


def _factor(ids):
    for i in ids:
        _DEC.local_solver(i)
    return len(ids)


def _solve(i, source, incoming):
    """Local solve of subdomain i (Eq. subPbm) in its owner."""
    return _DEC.local_solve(i, source, incoming)


def _scatter(i, incoming):
    """Zero-source local solve of i and its outgoing data toward every neighbour
    (one block column of S, Section 3), in its owner."""
    u = _DEC.local_solve(i, None, incoming)
    return {j: _DEC.outgoing(i, j, u, incoming[j]) for j in _DEC.neighbours(i)}


class PoolSweeper(Sweeper):
    """:class:`Sweeper` whose local solves run in ``processes`` worker processes.

    ``args`` / ``kwargs`` are the arguments the workers pass to
    :class:`Decomposition` (the same as ``dec``'s).  Call :meth:`close` when done.
    """

    def __init__(self, dec, args, kwargs=None, processes=2):
        super().__init__(dec)
        ctx = mp.get_context("spawn")
        self.P = max(1, int(processes))
        self.pools = [ctx.Pool(1, initializer=_init, initargs=(tuple(args), dict(kwargs or {})))
                      for _ in range(self.P)]
        self.owner = {i: k % self.P for k, i in enumerate(dec.subdomains)}
        # every worker factors its own subdomains, all workers at once
        jobs = [self.pools[w].apply_async(_factor, ([i for i in dec.subdomains if self.owner[i] == w],))
                for w in range(self.P)]
        for j in jobs:
            j.get()

    def close(self):
        for p in self.pools:
            p.close()
            p.join()

    # the stages' independent local solves, dealt to their owners at once
    def _map(self, fn, jobs):
        res = [self.pools[self.owner[job[0]]].apply_async(fn, job) for job in jobs]
        return [r.get() for r in res]

    def _scatter_many(self, ids, x):
        dec = self.dec
        return dict(zip(ids, self._map(_scatter, [(i, dec.incoming_of(x, i)) for i in ids])))

    def scatter_from(self, i, x):
        return self._scatter_many([i], x)[i]

    def apply_S(self, x):
        y = self.dec.zero_trace()
        for i, outs in self._scatter_many(list(self.dec.subdomains), x).items():
            for j, v in outs.items():
                y[(j, i)] = v
        return y

    def apply_elementary(self, x, d, kind, restrict=None):
        dec = self.dec
        src_d, dst_d = (d - 1, d) if kind == "E" else (d, d - 1)
        if restrict is not None and (src_d not in restrict or dst_d not in restrict):
            return
        # every solve of the step reads x before any of them is added in (the serial
        # loop does the same: a step writes only diagonal dst_d and reads src_d)
        for i, outs in self._scatter_many(list(dec.on_diagonal(src_d)), x).items():
            for j, v in outs.items():
                if dec.diagonal(j) == dst_d:
                    x[(j, i)] = x[(j, i)] + v

    def lifting_traces(self, r):
        dec = self.dec
        b = dec.zero_trace()
        ids = list(dec.subdomains)
        for i, w in zip(ids, self._map(_solve, [(i, dec.restrict(r, i), {}) for i in ids])):
            for j in dec.neighbours(i):
                b[(j, i)] = dec.outgoing(i, j, w, np.zeros(dec.side_length(i, j)))
        return b

    def reconstruct(self, r, g):
        dec = self.dec
        z = np.zeros(dec.n * dec.n, dtype=np.complex128)
        ids = list(dec.subdomains)
        for i, u in zip(ids, self._map(_solve, [(i, dec.restrict(r, i), dec.incoming_of(g, i)) for i in ids])):
            dec.insert(z, i, u)
        return z
