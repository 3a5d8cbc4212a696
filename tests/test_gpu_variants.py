"""Kernel variants kept as build options, checked on the GPU.

The default build runs the mixed mode's colour sum on the tensor cores from
120 flows, the crossover measured on GB300.  The 24-flow tensor-core form of
the table kernel (gg -> t t~ g g: tcgen05.mma of the CTA's 128 helicity rows
against the exact BF16 colour numerators, result in TMEM) stays available as
a build option (ME_MIXED_TC_MIN_NCOL=24).  This test builds that variant for
gg -> t t~ g g alone into a scratch directory, evaluates it in a child
process through the C ABI, and compares it with the FP64 oracle within the
FP32 tolerances (median <= 1e-5, maximum <= 1e-3) on a ragged batch.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LOW_MEDIAN, LOW_MAX = 1e-5, 1e-3

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2507_21039_gb300 as me
from paper_2507_21039_gb300 import build
build.build()
mom = np.load(sys.argv[2])
h = me.workload_handle("gg_ttxgg", "mixed")
out = me.me_sigmakin(h, torch.from_numpy(mom).cuda()).cpu().numpy()
h.close()
np.save(sys.argv[3], out)
"""


def test_table_kernel_tcgen05_colour_sum_variant(orc, tmp_path):
    w = WORKLOADS["gg_ttxgg"]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 517, w.cut_mask, PT_MIN, DR_MIN)
    ref = orc.me2("gg_ttxgg", mom, mt=MT, alpha=w.alpha)
    np.save(tmp_path / "mom.npy", mom)
    env = dict(os.environ, ME_BUILD_DIR=str(tmp_path / "build"), ME_LIBRARY=str(tmp_path / "build" / "libme.so"),
               ME_BUILD_PROCESSES="gg_ttxgg",
               ME_NVCC_EXTRA="-DME_MIXED_TC_MIN_NCOL=24 -DME_TAB_TC_UMMA=1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "mom.npy"), str(tmp_path / "out.npy")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(tmp_path / "out.npy")
    rel = np.abs(got / ref - 1)
    assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX, (np.median(rel), rel.max())
