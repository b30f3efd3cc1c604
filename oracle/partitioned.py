"""Oracle: one part of a partitioned LTS run with face-local messages (test infrastructure).

Sec. V-C: an element whose face neighbour lives in another memory space does not receive
that neighbour's buffer; the neighbour's side multiplies the buffer it would have sent by
the flux matrix F-_{j,h} of the shared face and sends only the 9 x F result H. The part
that owns the receiving element then applies the flux of its face to H.

`PartRun` turns an oracle `Solver` into one such part: the solver updates only the
elements of its part, and before every neighbour pass of cluster l it
* forms H = X F-_{j,h} for each face it sends whose receiver is in cluster l, with X the
  buffer the receiver would read (B1 for the same cluster; B3 if the sending element is
  the finer one; B2 in the first and B1 - B2 in the second half of the sending, coarser
  element's step) and (j, h) the sending element's face and orientation;
* hands the messages to `exchange(out, sources)` (out: destination part -> H rows; returns
  source part -> H rows), in the order of the exchange plan;
* uses the received H for its own cut faces.

The exchange plan is a table of rows (receiving element, receiving face, sending element,
sending face j, orientation h, receiving part, sending part, receiver cluster), ordered by
(receiving part, sending part, receiver cluster, receiving element, face), so both sides
of a message list its faces in the same order.
"""
import numpy as np


class PartRun:
    def __init__(self, solver, part, rank, plan, exchange):
        self.s = solver
        self.part = np.asarray(part)
        self.rank = int(rank)
        plan = np.asarray(plan, dtype=np.int64).reshape(-1, 8)
        self.recv_rows = plan[plan[:, 5] == rank]
        self.send_rows = plan[plan[:, 6] == rank]
        self.exchange = exchange
        solver.owned = self.part == rank
        solver.remote_h = self._remote

    def _message(self, rows, l, n):
        s = self.s
        H = np.zeros((len(rows), 9, s.basis.nf))
        for q, row in enumerate(rows):
            ks, js, hs = int(row[2]), int(row[3]), int(row[4])
            cs = s.clusters[ks]
            if cs == l - 1:
                X = s.B3[ks]
            elif cs == l + 1:
                X = s.B2[ks] if n % 2 == 0 else s.B1[ks] - s.B2[ks]
            else:
                X = s.B1[ks]
            H[q] = X @ s.basis.Fb[js][hs]
        return H

    def _remote(self, l, n, idx):
        send = self.send_rows[self.send_rows[:, 7] == l]
        out = {}
        for dst in np.unique(send[:, 5]):
            out[int(dst)] = self._message(send[send[:, 5] == dst], l, n)
        recv = self.recv_rows[self.recv_rows[:, 7] == l]
        got = self.exchange(out, sorted(set(int(x) for x in recv[:, 6])))
        if len(idx) == 0:
            return None
        pos = {int(e): p for p, e in enumerate(idx)}
        given = []
        for i in range(4):
            mask = np.zeros(len(idx), dtype=bool)
            H = np.zeros((len(idx), 9, self.s.basis.nf))
            for src in got:
                rows = recv[recv[:, 6] == src]
                for q, row in enumerate(rows):
                    if int(row[1]) == i:
                        p = pos[int(row[0])]
                        mask[p] = True
                        H[p] = got[src][q]
            given.append((mask, H[mask]) if np.any(mask) else None)
        return given
