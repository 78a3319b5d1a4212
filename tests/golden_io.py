"""Parser for the small text fixtures under tests/golden/ (each file cites its paper passage)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Returns dict(params={key: int}, tasks=[(name, kind, args...)], edges=[(a, b)],
    reach=[(a, b)], noreach=[(a, b)])."""
    out = dict(params={}, tasks=[], edges=[], reach=[], noreach=[])
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "task":
                out["tasks"].append(tuple(tok[1:]))
            elif tok[0] in ("edge", "reach", "noreach"):
                out[tok[0] if tok[0] != "edge" else "edges"].append((tok[1], tok[2]))
            else:
                out["params"][tok[0]] = int(tok[1])
    return out
