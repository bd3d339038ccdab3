"""Parsers for the worked examples under tests/golden/ (shared by the oracle
pins and the GPU parity tests; no method arithmetic here)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STATUS = {"MISS": 0, "FOUND": 1, "INSERTED": 2, "FULL": 3, "BAD_KEY": 4, "TIMEOUT": 5}
UPSERT_OPS = {"insert": -1, "add": 0, "max": 1, "replace": 2}


def api_semantics():
    """Yields ('count', None, None, n) or (op, key, val, (status, value))."""
    steps = []
    with open(os.path.join(GOLDEN, "api_semantics.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = (s.strip() for s in line.split("->"))
            parts = lhs.split()
            exp = rhs.split()
            if parts[0] == "count":
                steps.append(("count", None, None, int(exp[0])))
                continue
            op, key = parts[0], int(parts[1])
            val = int(parts[2]) if len(parts) > 2 else 0
            st = STATUS[exp[0]]
            value = int(exp[1]) if len(exp) > 1 else None
            steps.append((op, key, val, (st, value)))
    return steps


def run_api_semantics(table):
    """Replays api_semantics.txt on ``table`` (any object with single-batch
    methods insert/upsert/query/erase/count that take python lists and
    return (status list, value list)); returns a list of mismatch strings."""
    errs = []
    for i, (op, key, val, exp) in enumerate(api_semantics()):
        if op == "count":
            got = table.count()
            if got != exp:
                errs.append(f"step {i}: count {got} != {exp}")
            continue
        if op in UPSERT_OPS:
            st, _ = table.upsert([key], [val], UPSERT_OPS[op])
            got = (st[0], None)
        elif op == "query":
            st, v = table.query([key])
            got = (st[0], v[0])
        elif op == "erase":
            st, v = table.erase([key])
            got = (st[0], v[0])
        else:
            raise ValueError(op)
        want_st, want_v = exp
        if got[0] != want_st or (want_v is not None and got[1] != want_v):
            errs.append(f"step {i}: {op} {key} {val}: got {got}, want {exp}")
    return errs
