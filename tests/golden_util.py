"""Reader for the paper-transcribed expression tables under tests/golden/."""
import math
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table(name):
    """Return {symbol: expression string} from a golden file ('#' starts a comment)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, expr = line.split("=", 1)
            out[key.strip()] = expr.strip()
    return out


def evaluate(expr, **env):
    """Evaluate one arithmetic expression of a golden table with the given symbol values."""
    return float(eval(expr, {"__builtins__": {}, "math": math}, dict(env)))
