"""Host-side summary of an access matrix (Fig. 5), on hand-made counts (CPU only)."""
import torch

from paper_2110_01409_gb300 import dag


def test_locality_summary_hand_counts():
    c = torch.tensor([[6, 2, 0, 0],
                      [1, 1, 1, 1],
                      [0, 0, 0, 8],
                      [0, 0, 0, 0]], dtype=torch.int64)
    s = dag.locality(c)
    assert s["workers"] == 4
    assert abs(s["diag_share"] - 7 / 20) < 1e-15
    # own shares 0.75, 0.25, 0, 0 (an empty row counts as 0): two rows reach 1/4
    assert s["marked_rows"] == 2
    assert abs(s["own_share_median"] - 0.0) < 1e-15
