"""Critical density of the KA model on the Bethe lattice (section 4.2).

On a tree of branching k = z - 1 the probabilities that a site is (Y) occupied
and blocked, (B) empty and blocked so that particles below can never move up
to it, (F) occupied and frozen for the layer above, obey a recursion from one
layer to the next.  For k = 5 (z = 6) and m = 3 it reads

    Y' = F + 10 rho Y^3 [(1 - Y)^2 - B^2]
    B' = (1 - rho) F^4 (5 - 4 F)
    F' = rho [(Y + B)^5 + 5 Y^4 (1 - Y - B)]

and rho_c is the smallest density at which a fixed point other than (0, 0, 0)
exists.  Plain iteration of the map does not settle on the upper branch of
fixed points (it oscillates well above rho_c), so the branch is followed by
Newton's method from rho near 1 downwards until it ends; where it ends, in a
saddle-node, the fixed-point equations have a singular Jacobian, and the
system {x = step(x, rho), det(J - I) = 0} in the four unknowns (Y, B, F, rho)
is solved from the last point of the branch.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import fsolve


def step(v, rho: float) -> np.ndarray:
    """One layer of the recursion (k = 5, m = 3); v = (Y, B, F)."""
    y, b, f = v
    return np.array([f + 10.0 * rho * y ** 3 * ((1.0 - y) ** 2 - b * b),
                     (1.0 - rho) * f ** 4 * (5.0 - 4.0 * f),
                     rho * ((y + b) ** 5 + 5.0 * y ** 4 * (1.0 - y - b))])


def jacobian(v, rho: float) -> np.ndarray:
    """d step / d (Y, B, F)."""
    y, b, f = v
    return np.array([
        [10.0 * rho * (3.0 * y * y * ((1.0 - y) ** 2 - b * b) - 2.0 * y ** 3 * (1.0 - y)),
         -20.0 * rho * y ** 3 * b, 1.0],
        [0.0, 0.0, 20.0 * (1.0 - rho) * f ** 3 * (1.0 - f)],
        [rho * (5.0 * (y + b) ** 4 + 20.0 * y ** 3 * (1.0 - y - b) - 5.0 * y ** 4),
         5.0 * rho * ((y + b) ** 4 - y ** 4), 0.0]])


def fixed_point(rho: float, guess) -> tuple[np.ndarray, bool]:
    """Newton's method for x = step(x, rho) from guess; ok when it converged to a
    non-trivial point with every probability in [0, 1]."""
    x, _, ier, _ = fsolve(lambda v: step(v, rho) - v, np.asarray(guess, float),
                          fprime=lambda v: jacobian(v, rho) - np.eye(3), full_output=True,
                          xtol=1e-12)
    ok = (ier == 1 and np.abs(step(x, rho) - x).max() < 1e-10 and x[0] + x[2] > 1e-3
          and (x > -1e-9).all() and (x < 1.0 + 1e-9).all())
    return x, bool(ok)


def critical_density(rho_start: float = 0.99, drho: float = 0.002):
    """(rho_c, Y_c, B_c, F_c) where the upper branch of fixed points ends."""
    rho, x = rho_start, np.array([rho_start, 1.0 - rho_start, rho_start])
    last = None
    while rho > 0.5:
        y, ok = fixed_point(rho, x)
        if not ok:
            break
        last, x = (rho, y), y
        rho -= drho
    if last is None:
        raise RuntimeError("no non-trivial fixed point at the starting density")

    def saddle_node(u):
        v, r = u[:3], u[3]
        return np.concatenate([step(v, r) - v, [np.linalg.det(jacobian(v, r) - np.eye(3))]])

    u = fsolve(saddle_node, np.concatenate([last[1], [last[0]]]), xtol=1e-13)
    if np.abs(saddle_node(u)).max() > 1e-10:
        raise RuntimeError("the saddle-node system did not converge")
    return float(u[3]), float(u[0]), float(u[1]), float(u[2])


if __name__ == "__main__":
    print(critical_density())
