"""Plain FP64 CPU oracle for the l1-regularised least-squares hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls into it and shares no code with it: the two sides are
independent implementations of the same definitions, compared element by element.

What it computes (Fountoulakis & Gondzio, "Performance of First- and Second-Order
Methods for l1-Regularized Least Squares Problems"):

* ``rng``        -- counter-based SplitMix64 streams (Steele, Lea & Flood 2014); the
                    paper draws "uniformly at random" without naming a generator.
* ``generator``  -- Procedure IGen (Sec. 3.1), Procedure IGen2 (Sec. 3.2), the
                    construction A = (P1 G~ P2) Sigma G^T of Eq. (bd8) with the Givens
                    stages of Sec. 4.1-4.2, and Procedure OsGen (Sec. 6).
* ``operators``  -- Algorithms MvPA and MvPAt (Sec. 4), matrix-free products.
* ``solvers``    -- the objective of Eq. (prob1), a duality-gap certificate, FISTA
                    (Sec. 8.1) and pdNCG (Newton-CG on the pseudo-Huber smoothing,
                    Eqs. (pseudoHuber), (prob2), (bd4), Sec. 8.1 and 8.3).
* ``brute``      -- brute-force support enumeration for tiny n (the restricted
                    stationarity system of Sec. 3.2, Eq. (bd9)).

Every function is pinned by a ``-m "not gpu"`` test against something other than
itself (printed counts, closed forms, optimality conditions, brute force).  Where a
function has no such pin its docstring says "parity unpinned".
"""

from . import rng, generator, operators, solvers, brute  # noqa: F401
