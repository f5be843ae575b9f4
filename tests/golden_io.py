"""Reader for the hand-derived fixtures in tests/golden/ (``key v1 v2 ...``
lines; values may be fractions like 225/11; '#' starts a comment)."""
import os
from fractions import Fraction

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            nums = [float(Fraction(v)) for v in vals]
            out[key] = nums[0] if len(nums) == 1 else nums
    return out
