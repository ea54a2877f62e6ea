"""The precomputed metric geometry of asterx_prepare against the oracle's interpolation, bit for bit.

asterx_prepare evaluates the 4th-order tensor-product stencils of Sec. 3.2 separably (an x pass into workspace
scratch, then y and z contractions per column), with rounded multiply and add in the same order as the oracle's
per-point sums (x innermost, then y, then z).  The records must therefore equal the oracle's values exactly:
the recovery's atmosphere test compares D~ with sqrt(gamma) rho_atm, and identical inputs must decide
identically on both sides.  White-box: the test reads the records from the workspace in the layout of
csrc/layout.h (centre record of 53 fields at the workspace start, then three face records of 15 fields, each
group at pitch V and 256-byte aligned field stride).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import GpuCase
from paper_2406_11669_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCG, NFG = 53, 15
CG_DALP = 23
FG_GUDD, FG_SQG, FG_IALP, FG_ISQG, FG_WIDTH = 10, 11, 12, 13, 14
SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def records(case):
    s = case.solver
    V = int(np.prod(case.w.shape))
    fs = (V + 31) // 32 * 32
    off = s.ws_ptr.value - s.ws.data_ptr()
    buf = s.ws[off:off + (NCG + 3 * NFG) * fs * 8].view(torch.float64).cpu().numpy()
    cg = np.stack([buf[q * V:(q + 1) * V].reshape(case.w.shape) for q in range(NCG)])
    fg = [np.stack([buf[NCG * fs + (d * NFG + q) * V:NCG * fs + (d * NFG + q + 1) * V].reshape(case.w.shape)
                    for q in range(NFG)]) for d in range(3)]
    return cg, fg


def cells(w):
    N = w.N
    return (slice(0, N[2]), slice(0, N[1]), slice(0, N[0]))


def inner_cells(w):
    g, n = w.g, w.n
    return (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))


def faces(w, d):
    N = list(w.N)
    N[d] += 1
    return (slice(0, N[2]), slice(0, N[1]), slice(0, N[0]))


def check_exact(case, M):
    w = case.w
    cg, fg = records(case)
    ref = O.centre_metric(w, M)
    sl = cells(w)
    for q in range(CG_DALP):
        assert np.array_equal(cg[q][sl], ref[q][sl]), ("centre", q)
    isl = inner_cells(w)
    outside = np.zeros(w.shape, bool)
    outside[sl] = True
    outside[isl] = False  # padded cells outside the interior: derivatives are not used there and are zero
    for q in range(CG_DALP, NCG):
        assert np.array_equal(cg[q][isl], ref[q][isl]), ("centre derivative", q)
        assert np.all(cg[q][outside] == 0.0)
    for d in range(3):
        fr = O.face_metric(w, M, d)
        fsl = faces(w, d)
        for q in range(10):
            assert np.array_equal(fg[d][q][fsl], fr[q][fsl]), ("face", d, q)
        assert np.array_equal(fg[d][FG_GUDD][fsl], fr[10 + SYM[d][d]][fsl])
        assert np.array_equal(fg[d][FG_SQG][fsl], fr[16][fsl])
        assert np.array_equal(fg[d][FG_IALP][fsl], 1.0 / fr[0][fsl])
        assert np.array_equal(fg[d][FG_ISQG][fsl], 1.0 / fr[16][fsl])
        assert np.array_equal(fg[d][FG_WIDTH][fsl], fr[0][fsl] * np.sqrt(fr[10 + SYM[d][d]][fsl]))


@pytest.mark.parametrize("name", ["smooth_general", "star", "balsara_schwarzschild"])
def test_prepared_geometry_equals_the_oracle_exactly(name):
    need_gpu()
    w = {"smooth_general": W.smooth_general(n=(9, 7, 11)),
         "star": W.star_block((16, 20, 12), (0.3515625, -0.0390625, -0.0234375), name="star_block"),
         "balsara_schwarzschild": W.balsara_schwarzschild(n=(26, 10, 9))}[name]
    case = GpuCase(w)
    check_exact(case, case.M)


def test_reprepare_with_another_metric():
    """A second prepare from a different metric (as every stage of a time-dependent metric does) leaves no trace
    of the first."""
    need_gpu()
    w = W.smooth_general(n=(8, 9, 7))
    case = GpuCase(w)
    M2 = case.M.copy()
    M2[0] *= 1.05
    M2[2] += 0.01
    M2[5] += 0.003
    case.solver.prepare(case.dev(M2))
    check_exact(case, M2)
