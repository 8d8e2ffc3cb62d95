"""Reader for tests/golden/closed_forms.txt (textbook closed forms)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_forms.txt")


def closed_form(name: str, kin: str = "-"):
    """{order: complex} for one integral at one kinematic point."""
    out = {}
    with open(_PATH) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            body = line.split("#")[0].split()
            if body[0] == name and body[1] == kin:
                out[int(body[2])] = complex(float(body[3]), float(body[4]))
    if not out:
        raise KeyError((name, kin))
    return out
