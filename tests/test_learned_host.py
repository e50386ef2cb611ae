"""Host side of the learned guess: the network's sizes agree between the
header, the binding and the oracle, and the initial parameters are
Glorot-uniform weights with zero biases in the library's order
(W1, b1, W2, b2, W3, b3, each W row-major [fan_out][fan_in])."""
import os
import re

import numpy as np

from oracle import mlp as om
from paper_2105_01722_gb300 import gdg, learned

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sizes_agree_everywhere():
    sizes = (gdg.MLP_IN, gdg.MLP_HID, gdg.MLP_HID, gdg.MLP_OUT)
    assert sizes == (162, 64, 64, 81) and tuple(om.SIZES) == sizes
    nw = sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    assert gdg.MLP_NWEIGHT == nw and gdg.MLP_NPARAM == nw + sum(sizes[1:])
    header = open(os.path.join(ROOT, "include", "gdg.h")).read()
    for name, value in (("GDG_MLP_IN", gdg.MLP_IN), ("GDG_MLP_HID", gdg.MLP_HID), ("GDG_MLP_OUT", gdg.MLP_OUT),
                        ("GDG_MLP_NPARAM", gdg.MLP_NPARAM), ("GDG_MLP_NWEIGHT", gdg.MLP_NWEIGHT)):
        m = re.search(r"%s\s*=\s*(\d+)" % name, header) or re.search(r"#define\s+%s\s+(\d+)" % name, header)
        assert m and int(m.group(1)) == value, name


def test_glorot_initial_parameters():
    P = learned.glorot_params(3)
    assert P.dtype == np.float32 and P.size == gdg.MLP_NPARAM
    assert np.array_equal(P, learned.glorot_params(3)) and not np.array_equal(P, learned.glorot_params(4))
    sizes = (gdg.MLP_IN, gdg.MLP_HID, gdg.MLP_HID, gdg.MLP_OUT)
    ref = om.init_params(3, sizes)       # same seed, same draw order: same values
    o = 0
    for k, (fi, fo) in enumerate(zip(sizes[:-1], sizes[1:])):
        W = P[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = P[o:o + fo]
        o += fo
        lim = np.sqrt(6.0 / (fi + fo))
        assert np.abs(W).max() <= lim and np.abs(W).max() > 0.9 * lim
        assert abs(W.std() - lim / np.sqrt(3.0)) < 0.05 * lim / np.sqrt(3.0)   # uniform on [-lim, lim]
        assert not b.any()
        assert np.allclose(W, ref[2 * k].astype(np.float32)) and not ref[2 * k + 1].any()
    assert o == P.size
