"""Reader for the paper-printed values in paper_section3_table1.txt."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_section3_table1.txt")


def values():
    out = {}
    for line in open(_PATH):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, v = (s.strip() for s in line.split("=", 1))
        parts = v.split()
        conv = []
        for p in parts:
            try:
                conv.append(float(p))
            except ValueError:
                conv.append(p)
        out[k] = conv[0] if len(conv) == 1 else conv
    return out
