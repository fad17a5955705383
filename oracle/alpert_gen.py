"""Generator of the oracle's Alpert log-singular end-correction table.

TEST INFRASTRUCTURE ONLY: nothing in the product imports this module.

The paper (Sec. 4.1, hybrid Gauss-trapezoid rule of order 10; Alpert 1999) does
not print the correction nodes and weights, so they are solved for here from
the moment conditions that define the rule.  For a function f(x) = phi(x) +
psi(x) log(x) on [0, inf) (phi, psi smooth) the corrected trapezoid sum

    h * sum_{k=1..j} w_k f(x_k h)  +  h * sum_{i>=a} f(i h)

reproduces the integral to O(h^j log h) when, for p = 0..j-1,

    sum_k w_k x_k^p          = -zeta(-p, a)          (smooth part)
    sum_k w_k x_k^p log x_k  =  zeta'(-p, a)         (log part)

where zeta(s, a) is the Hurwitz zeta function and ' is d/ds.  (Both follow
from the zeta-regularised Euler-Maclaurin expansion of the shifted
trapezoid sum: sum_{i>=a} (ih)^p = h^p zeta(-p, a), and the log h terms
cancel by the first set.)

The 2j equations are solved by Newton's method along a homotopy from an
arbitrary positive starting rule (moments interpolated linearly towards the
targets), in 60-digit arithmetic.  Output: `alpert_log_j10_a10.txt`, one
"x_k w_k" pair per line, 30 significant digits.

Run:  python -m oracle.alpert_gen
"""
import os

import mpmath as mp


def _moments(x, w, j):
    rows = [mp.fsum(w[k] * x[k] ** p for k in range(j)) for p in range(j)]
    rows += [mp.fsum(w[k] * x[k] ** p * mp.log(x[k]) for k in range(j)) for p in range(j)]
    return mp.matrix(rows)


def _jacobian(x, w, j):
    # unknowns: (log x_1..log x_j, w_1..w_j); d/d(log x) = x d/dx
    J = mp.matrix(2 * j, 2 * j)
    for p in range(j):
        for k in range(j):
            lx = mp.log(x[k])
            xp = x[k] ** p
            J[p, k] = w[k] * p * xp
            J[p, j + k] = xp
            J[j + p, k] = w[k] * (p * xp * lx + xp)
            J[j + p, j + k] = xp * lx
    return J


def targets(j, a):
    """Right-hand sides of the moment conditions (Hurwitz zeta values)."""
    smooth = [-mp.zeta(-p, a) for p in range(j)]
    logp = [mp.zeta(-p, a, derivative=1) for p in range(j)]
    return mp.matrix(smooth + logp)


def solve_rule(j, a, dps=60, gamma=2.0):
    """Nodes and weights (sorted by node) of the j-point log rule with skip a."""
    with mp.workdps(dps):
        tgt = targets(j, a)
        x = [mp.mpf(a) * mp.mpf((k + 0.5) / j) ** gamma for k in range(j)]
        w = [mp.mpf(a) / j * gamma * mp.mpf((k + 0.5) / j) ** (gamma - 1) for k in range(j)]
        b0 = _moments(x, w, j)
        u = [mp.log(t) for t in x] + w
        lam, dl = mp.mpf(0), mp.mpf("0.01")
        tol = mp.mpf(10) ** (-(dps - 15))
        while lam < 1:
            l2 = min(mp.mpf(1), lam + dl)
            rhs = b0 * (1 - l2) + tgt * l2
            v, ok = list(u), False
            for _ in range(40):
                xx = [mp.exp(t) for t in v[:j]]
                ww = v[j:]
                r = _moments(xx, ww, j) - rhs
                if mp.norm(r) < tol:
                    ok = True
                    break
                try:
                    d = mp.lu_solve(_jacobian(xx, ww, j), -r)
                except ZeroDivisionError:
                    break
                if mp.norm(d) > 1:
                    break
                v = [v[i] + d[i] for i in range(2 * j)]
            if ok:
                u, lam, dl = v, l2, min(dl * mp.mpf("1.5"), mp.mpf("0.2"))
            else:
                dl /= 4
                if dl < mp.mpf("1e-12"):
                    raise RuntimeError("homotopy failed for j=%d a=%d" % (j, a))
        x = [mp.exp(t) for t in u[:j]]
        w = u[j:]
        return sorted(zip(x, w))


TABLE = os.path.join(os.path.dirname(__file__), "alpert_log_j10_a10.txt")


def main():
    rule = solve_rule(10, 10)
    with open(TABLE, "w") as f:
        f.write("# Alpert log-singular end correction, j=10 nodes, skip a=10 (order 10).\n")
        f.write("# Written by oracle/alpert_gen.py from the moment conditions; x_k w_k.\n")
        for xk, wk in rule:
            f.write("%s %s\n" % (mp.nstr(xk, 30), mp.nstr(wk, 30)))
    print("wrote", TABLE)


if __name__ == "__main__":
    main()
