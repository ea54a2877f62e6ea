"""Host checks of the seeded input generators that both sides consume (no method arithmetic here)."""
import os

import numpy as np

from paper_2406_11669_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "weak_field_gradient.txt")


def test_gradient_directions_cover_the_independent_entries_only():
    """Directions for the gradient checks: nonzero exactly on the independent entries of the perturbed fields
    (cells g..g+n-1; an edge field's vertex-like axes g..g+n-1 where periodic, g..g+n otherwise), never on p,
    reproducible from the seed, and named as the stored oracle values are."""
    for bc in (W.BC_PERIODIC, W.BC_COPY):
        w = W.smooth_general(n=(6, 5, 4), bc=bc)
        g, n = w.g, w.n
        dirs = W.gradient_directions(w)
        assert [d[0] for d in dirs] == list(W.GRADIENT_DIRECTIONS)
        for name, dP, dA in dirs:
            assert not dP[1].any()
            cells = np.zeros(w.shape, dtype=bool)
            cells[g:g + n[2], g:g + n[1], g:g + n[0]] = True
            for v in (0, 2, 3, 4):
                want = name in ("all_fields_a", "all_fields_b") or (name == "rho" and v == 0)
                assert np.array_equal(dP[v] != 0.0, cells & want), (name, v)
            for v in range(3):
                mask = np.zeros(w.shape, dtype=bool)
                hi = [g + n[a] + (0 if (a == v or bc == W.BC_PERIODIC) else 1) for a in range(3)]
                mask[g:hi[2], g:hi[1], g:hi[0]] = True
                want = name != "rho"
                assert np.array_equal(dA[v] != 0.0, mask & want), (name, v)
        again = W.gradient_directions(w)
        assert all(np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) for a, b in zip(dirs, again))
    with open(GOLDEN) as f:
        names = [line.split()[0] for line in f if line.strip() and not line.startswith("#")]
    assert names == list(W.GRADIENT_DIRECTIONS)
