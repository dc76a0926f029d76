"""Reader of the fixtures under tests/golden/: `key = value` lines (numbers),
'#' comments holding the citation of each file."""
import pathlib

GOLDEN = pathlib.Path(__file__).resolve().parent / "golden"


def load(name):
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, value = (s.strip() for s in line.split("=", 1))
        out[key] = float(value)
    return out
