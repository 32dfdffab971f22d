"""Static check of the programmatic dependent launches (no GPU needed).

A kernel launched with launch_pdl may be scheduled before the kernel ahead of it on the stream has
finished; it is correct only if its first statement is pdl_enter() (griddepcontrol.wait).  This
test finds every launch_pdl call in the CUDA sources and checks the launched kernel's definition."""
import pathlib
import re

CSRC = pathlib.Path(__file__).resolve().parent.parent / "paper_2607_25330_b300" / "csrc"


def _kernel_bodies(text):
    """name -> list of first statements of its __global__ definitions."""
    out = {}
    for m in re.finditer(r"__global__\s", text):
        j = text.index("{", m.end())
        sig = text[m.end():j]
        names = [n for n in re.findall(r"(\w+)\s*\(", sig) if n.startswith("k_")]
        if not names:
            continue
        first = text[j + 1:].lstrip().split(";", 1)[0].strip()
        out.setdefault(names[0], []).append(first)
    return out


def test_every_pdl_launched_kernel_waits_first():
    srcs = {p.name: p.read_text() for p in CSRC.glob("*.cu")}
    kernels = {}
    for text in srcs.values():
        for k, v in _kernel_bodies(text).items():
            kernels.setdefault(k, []).extend(v)
    launched = set()
    for name, text in srcs.items():
        for m in re.finditer(r"launch_pdl\(\s*(\w+)", text):
            launched.add(m.group(1))
    assert len(launched) >= 20, launched
    for k in sorted(launched):
        assert k in kernels, f"launch_pdl of {k}: no __global__ definition found"
        for first in kernels[k]:
            assert first == "pdl_enter()", f"{k} starts with `{first}`, not pdl_enter()"


def test_pdl_enter_waits_on_the_predecessor():
    text = (CSRC / "pdl.cuh").read_text()
    body = text[text.index("void pdl_enter()"):]
    body = body[:body.index("}")]
    assert "griddepcontrol.wait" in body
    assert "cudaLaunchAttributeProgrammaticStreamSerialization" in text
