"""Parity where the method itself is discontinuous.

The Sec. 2.3 separation rule (the oracle's and the library's SEP23 flag) takes
W = Delta where Delta v . n > 0 and W = 0 elsewhere: a step at Delta v . n = 0.
The series drives the particles of an active contact towards that surface, so
two correct evaluations of the same step that differ only in rounding can take
opposite sides of it at a few particles, and their results then differ by those
particles' share of Delta, not by a rounding error.  (The Sec. 2.4 cone rule
has no such step: its projection is continuous.)

`envelope` measures this with the FP64 oracle alone: it moves the inputs v and C
by `eps` relative (seeded normal factors, a few trials) and returns, element by
element, the largest change of the oracle's own outputs.  A GPU result is then
held to the FP32 tolerance plus that envelope, element by element: particles
away from the step keep the plain tolerance, and only where a rounding-level
change of the inputs already moves the oracle is the comparison widened, by
exactly what the oracle showed.  eps = 1e-6 is about ten FP32 units in the last
place, more than the relative rounding error of the FP32 path's inputs to the
step's decision.
"""
import numpy as np


def envelope(run, v, C, eps=1e-6, trials=4, seed=0):
    """run(v, C) -> (v_out, C_out) with everything else fixed.  Returns
    (reference v_out, reference C_out, envelope of v_out, envelope of C_out)."""
    v0, C0 = run(v, C)
    ev, eC = np.zeros_like(v0), np.zeros_like(C0)
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        v1, C1 = run(v * (1 + eps * rng.standard_normal(v.shape)), C * (1 + eps * rng.standard_normal(C.shape)))
        ev = np.maximum(ev, np.abs(v1 - v0))
        eC = np.maximum(eC, np.abs(C1 - C0))
    return v0, C0, ev, eC


def excess(got, ref, env, tol_abs):
    """Largest |got - ref| - env over the elements, in units of tol_abs (a
    value <= 1 passes).  Shapes of got, ref and env agree."""
    d = np.abs(np.asarray(got, dtype=np.float64) - ref) - env
    return max(float(d.max()), 0.0) / tol_abs
