import os

HERE = os.path.dirname(os.path.abspath(__file__))


def printed_values():
    """key -> (value, unit, citation) from paper_printed_values.txt"""
    out = {}
    with open(os.path.join(HERE, "paper_printed_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val, unit, cite = line.split(None, 3)
            out[key] = (float(val), unit, cite)
    return out
