"""Small shared test helpers (no scheme arithmetic)."""
import os
import re

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(path=None):
    """Names of the functions declared in include/*.h."""
    names = []
    paths = [path] if path else sorted(
        os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
        if f.endswith(".h"))
    for p in paths:
        text = open(p).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


def rel_errors(a, ref):
    """Per variable (relative L2, relative Linf) of a against ref, both
    [B][C][ny][nx]; a variable that is zero in ref is normalised by the
    largest magnitude of variable 0."""
    a = torch.as_tensor(a, dtype=torch.float64).cpu()
    ref = torch.as_tensor(ref, dtype=torch.float64).cpu()
    out = []
    s0 = float(ref[:, 0].abs().max())
    for c in range(ref.shape[1]):
        d = a[:, c] - ref[:, c]
        n2 = float(ref[:, c].norm())
        ninf = float(ref[:, c].abs().max())
        if ninf == 0.0:
            n2 = s0 * ref[:, c].numel() ** 0.5
            ninf = s0
        out.append((float(d.norm()) / n2, float(d.abs().max()) / ninf))
    return out


def f32(q):
    return torch.as_tensor(np.asarray(q, dtype=np.float32))
