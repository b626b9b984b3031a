"""CPU pin of the oracle's sweep against a restatement from scratch.

A few sweeps of a tiny problem are written out here move by move from the method's definition
(Sec. 2.2: the two-bin move that keeps both sum rules, the positivity factor and the Metropolis
test of Eq. probability-density) and the conventions the library documents: Philox4x32-10 from
its published round structure (Salmon et al., SC'11) with counter (move, sweep, walker, 0) and
the 64-bit seed as key; words 0 and 1 choose the bins, word 2 the amplitude, word 3 the
acceptance draw, a word w read as (w + 1/2) 2^-32; the amplitude heuristic y = min(1, a)^2 from
the previous sweep's acceptance a with a floor 1e-4; the geometric schedule in units of the
start residue.  Unlike the oracle, chi2 is recomputed from scratch after every move.  The
oracle must take the same decisions (its FNV hash of move outcomes and its accepted counts) and
end in the same spectra.
"""
import numpy as np

import oracle as O
from workloads import Peak, make_problem

M32 = 0xFFFFFFFF


def philox(ctr, key):
    x = [int(v) & M32 for v in ctr]
    k = [key & M32, (key >> 32) & M32]
    for r in range(10):
        if r:
            k = [(k[0] + 0x9E3779B9) & M32, (k[1] + 0xBB67AE85) & M32]
        p0, p1 = 0xD2511F53 * x[0], 0xCD9E8D57 * x[2]
        x = [((p1 >> 32) ^ x[1] ^ k[0]) & M32, p1 & M32, ((p0 >> 32) ^ x[3] ^ k[1]) & M32, p0 & M32]
    return x


def unit(w):
    return (w + 0.5) * 2.0 ** -32


def run_by_definition(P, n_walkers, n_sweeps, T_start, T_end, move_scale, seed):
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)   # pinned against quadrature elsewhere
    a0, _ = O.initial_spectrum(P.omega, P.A, P.B)        # pinned by its sum rules elsewhere
    x, A, B, N = P.omega, P.A, P.B, P.n_omega
    chi2_of = lambda a: float(np.sum((Fh - K @ a) ** 2))
    chi2_0 = chi2_of(a0)
    out_a, out_hash, out_acc = [], [], np.zeros((n_sweeps, n_walkers), dtype=int)
    for w in range(n_walkers):
        a = a0.copy()
        chi2 = chi2_0
        h = 0xCBF29CE484222325
        acc_prev = N
        for n in range(n_sweeps):
            T = chi2_0 * T_start * (T_end / T_start) ** (n / (n_sweeps - 1))
            y = max(min(1.0, acc_prev / N) ** 2, 1e-4)
            acc = 0
            for mv in range(N):
                w0, w1, w2, w3 = philox((mv, n, w, 0), seed)
                p = (w0 * N) >> 32
                s = (w1 * (N - 1)) >> 32
                s += s >= p
                eps = y * move_scale * (2.0 * unit(w2) - 1.0)
                r = 1.0 - eps
                dp = eps * (B - A * x[s]) / (x[p] - x[s])
                ds = eps * (B - A * x[p]) / (x[s] - x[p])
                ap, as_ = r * a[p] + dp, r * a[s] + ds
                if ap < 0.0 or as_ < 0.0:
                    code = 2
                else:
                    new = r * a
                    new[p], new[s] = ap, as_
                    c_new = chi2_of(new)
                    D = c_new - chi2
                    if D <= 0.0 or unit(w3) < np.exp(-D / T):
                        a, chi2, code = new, c_new, 1
                        acc += 1
                    else:
                        code = 0
                h = ((h ^ code) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
            out_acc[n, w] = acc
            acc_prev = acc
        out_a.append(a)
        out_hash.append(h)
    return np.array(out_a), np.array(out_hash, dtype=np.uint64), out_acc


def test_oracle_sweeps_are_the_definition():
    tau = 0.5 * np.arange(8, dtype=np.float64)
    P = make_problem("definition", tau, 12, 4.0, [Peak("lorentz", 1.5, 0.4, 0.7), Peak("gauss", 2.8, 0.3, 0.3)],
                     1e-3, 2, 4)
    kw = dict(n_sweeps=6, T_start=1.0, T_end=1e-2, move_scale=0.2, seed=0x1234_5678_9ABC)
    a_ref, h_ref, acc_ref = run_by_definition(P, 4, **kw)
    sched = O.Schedule(sweeps_per_block=1000, resync_every=1000, **kw)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 4, sched)
    acc, _, _ = an.run(trace=True)
    # decisions went every way: accepted, rejected by the test, rejected by positivity
    assert 0 < acc_ref.sum() < 6 * 4 * 12 and an.n_pos.sum() > 0
    np.testing.assert_array_equal(acc, acc_ref)
    np.testing.assert_array_equal(an.hash, h_ref)
    np.testing.assert_allclose(an.a, a_ref, rtol=1e-12, atol=1e-14 * np.abs(a_ref).max())
