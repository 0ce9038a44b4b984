"""An independent restatement of Listing 1 (Section 2) for tiny supernodes.

Used only to cross-check the oracle's bookkeeping on brute-force enumerations.
It is written differently from the oracle on purpose: nothing is ever moved.
The matrix stays in original order; a column is "eliminated" or not, and the
candidate order is the original index order of the uneliminated columns (the
stable shift of accepted pivots to the front never reorders the rest).  The
tests are written from eq. (2.1) and eq. (2.2) directly with a 2x2 inverse from
numpy; only the nonsingularity guard of test_2x2 is taken from the listing.
"""
import numpy as np


def restated_listing(A11, outer, u, small=1e-20, strict_abs=False):
    """Returns (order of eliminated columns, kinds) where kinds[c] is '1', '2a',
    '2b', 'z' or 'd' per original column c."""
    p = A11.shape[0]
    M = np.vstack([np.array(A11, float), np.array(outer, float).reshape(-1, p)])
    r = M.shape[0] - p
    elim = [False] * p
    order, kinds = [], ["d"] * p

    def live_rows(excl):
        rows = [i for i in range(p) if not elim[i] and i not in excl]
        return rows + list(range(p, p + r))

    def update(piv_cols):
        # D block and its inverse on the pivot columns
        Db = M[np.ix_(piv_cols, piv_cols)]
        Di = np.linalg.inv(Db) if len(piv_cols) == 2 else np.array([[1.0 / Db[0, 0]]])
        rest = [c for c in range(p) if not elim[c] and c not in piv_cols]
        old = M.copy()
        for k in rest:
            akq = old[k, piv_cols]
            for i in rest:
                M[i, k] = old[i, k] - old[i, piv_cols] @ Di @ akq
            for i in range(p, p + r):
                if strict_abs:
                    M[i, k] = old[i, k] + old[i, piv_cols] @ np.abs(Di) @ np.abs(akq)
                else:
                    M[i, k] = old[i, k] - old[i, piv_cols] @ Di @ akq

    def uneliminated():
        return [c for c in range(p) if not elim[c]]

    m_list = uneliminated()
    pos = 1 if p >= 2 else 0
    accepted = False
    while not all(elim):
        live = uneliminated()
        if pos >= len(live):
            if not accepted:
                break
            accepted, pos = False, 0
            continue
        m = live[pos]
        col = [abs(M[i, m]) for i in live_rows(())]
        if max(col) < small:
            elim[m] = True
            order.append(m)
            kinds[m] = "z"
            accepted = True
            continue  # next candidate is the column after m: same live index
        if pos > 0:
            before = live[:pos]
            vals = [abs(M[m, j]) for j in before]
            t = before[int(np.argmax(vals))]  # argmax returns the first maximiser
            maxt = max([abs(M[i, t]) for i in live_rows((t, m))], default=0.0)
            maxm = max([abs(M[i, m]) for i in live_rows((t, m))], default=0.0)
            att, atm, amm = M[t, t], M[t, m], M[m, m]
            amax = max(abs(att), abs(atm), abs(amm))
            ok = False
            if amax >= small:
                ds = 1.0 / amax
                d1 = (atm * ds) * atm
                d0 = amm * ds * att
                if abs(d0 - d1) > max(small, abs(d0) / 2, abs(d1) / 2):
                    if max(maxm, maxt) < small:
                        ok = True
                    else:
                        Dinv = np.linalg.inv(np.array([[att, atm], [atm, amm]]))
                        g = np.abs(Dinv) @ np.array([maxt, maxm])
                        ok = bool(np.all(g <= (1.0 / u) * (1 + 1e-13)))
            if ok:
                update([t, m])
                elim[t] = elim[m] = True
                order += [t, m]
                kinds[t], kinds[m] = "2a", "2b"
                accepted = True
                pos -= 1  # t, m left the live list before the next candidate
                continue
        maxm1 = max([abs(M[i, m]) for i in live_rows((m,))], default=0.0)
        if abs(M[m, m]) >= u * maxm1:
            update([m])
            elim[m] = True
            order.append(m)
            kinds[m] = "1"
            accepted = True
            continue
        pos += 1
    return order, kinds
