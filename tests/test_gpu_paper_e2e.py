"""The paper-shaped end-to-end report (Sec. 3 workflow on synthetic data):
structure and the invariants that must hold at any size — the topology fix
preserves every case, accuracies stay in [0, 1], and the compressed modes
stream fewer bytes than the raw field at the usual bounds."""
import pytest
import torch

from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import paper_e2e

pytestmark = pytest.mark.gpu


def test_paper_e2e_small():
    assert torch.cuda.is_available()
    chr_build.build()
    out = paper_e2e.run(size=64, reps=1, seed=7)
    assert set(out["modes"]) == {"fix", "translate_100", "translate_99", "translate_95", "translate_80"}
    assert out["modes"]["fix"]["topology_accuracy"] == 1.0
    for m in out["modes"].values():
        assert 0.0 <= m["topology_accuracy"] <= 1.0
        assert m["total_ms"] > m["stream_ms"] > 0
        assert abs(m["speedup_vs_raw"] - out["baseline"]["total_ms"] / m["total_ms"]) < 1e-9
    # looser accuracy never tightens the bound
    ebs = [out["modes"][k]["error_bound"] for k in ("translate_100", "translate_99", "translate_95", "translate_80")]
    assert ebs == sorted(ebs)
    assert out["modes"]["fix"]["compressed_bytes"] < out["baseline"]["bytes"]
