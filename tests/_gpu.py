"""Helpers for the GPU tests: numpy <-> CUDA tensors and the table's layout
parameters.  No method arithmetic here."""
import numpy as np

DESIGNS = [("double", False), ("double", True), ("p2", False), ("p2", True), ("iceberg", True)]
DESIGN_IDS = ["DoubleHT", "DoubleHT(M)", "P2HT", "P2HT(M)", "IcebergHT(M)"]


def dev(a, device="cuda"):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(device)


def host(t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if a.dtype == np.int64 else a


def layout_of(table):
    """Arguments of oracle.layout_check for a dumped table."""
    inf = table.info()
    slots, tags = table.dump()
    return dict(slots=slots.reshape(-1), tags=tags, nb=inf["buckets"], B=inf["bucket_slots"],
                scheme=inf["scheme"], pmax=inf["max_probe"], seed1=inf["seed1"], seed2=inf["seed2"])


def check_layout(oracle, table, expect_live=None):
    L = layout_of(table)
    r = oracle.layout_check(L["slots"], L["tags"], L["nb"], L["B"], L["scheme"], L["pmax"],
                            L["seed1"], L["seed2"])
    bad = {k: r[k] for k in ("bad_bucket", "duplicates", "tag_mismatch", "early_exit", "empty_not_suffix",
                             "resv") if r[k]}
    assert not bad, f"layout violations: {bad}"
    if expect_live is not None:
        assert r["live"] == expect_live, (r["live"], expect_live)
    return r, L
