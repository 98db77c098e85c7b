"""Static check of the programmatic-dependent-launch contract in the CUDA
sources: a kernel started through launch_pdl may become resident while its
predecessor in the stream still runs, so its first statement must be
pdl_wait() (which returns once the predecessor has completed and its writes
are visible).  Cooperative kernels are never launched that way."""
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_2506_04732_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu"):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = fh.read()
    return out


def _kernel_bodies(src, name):
    for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", src):
        i = src.index("{", m.end())
        if ";" in src[m.end():i]:
            continue  # a declaration
        yield src[i + 1:]


def test_every_pdl_launched_kernel_waits_first():
    srcs = _sources()
    launched = set()
    for s in srcs.values():
        launched |= set(re.findall(r"launch_pdl\(\s*([A-Za-z_][A-Za-z_0-9]*)", s))
        # cluster launches through cudaLaunchKernelEx with the programmatic
        # attribute: the stage kernels' cluster variants and the cluster QR
        launched |= set(re.findall(r"launch_stages\([^;]*?([A-Za-z_][A-Za-z_0-9]*)<true>", s))
        launched |= set(re.findall(r"cudaLaunchKernelEx\(&cfg,\s*([A-Za-z_][A-Za-z_0-9]*)", s))
    launched.discard("clus")  # launch_stages' parameter: its kernels are found above
    assert len(launched) >= 10
    for k in sorted(launched):
        bodies = [b for s in srcs.values() for b in _kernel_bodies(s, k)]
        assert bodies, f"kernel {k} not found"
        for b in bodies:
            assert b.lstrip().startswith("pdl_wait();"), f"{k} touches memory before pdl_wait()"


def test_cooperative_kernels_are_not_pdl_launched():
    srcs = _sources()
    coop = set()
    for s in srcs.values():
        coop |= set(re.findall(r"cudaLaunchCooperativeKernel\(\s*\(\s*(?:const\s+)?void\s*\*\s*\)\s*([A-Za-z_][A-Za-z_0-9]*)", s))
        # launch_stages(coop, cluster, ...): the first is launched cooperatively
        coop |= set(re.findall(r"launch_stages\(\s*([A-Za-z_][A-Za-z_0-9]*)<false>", s))
    coop.discard("coop")
    assert {"cholqr3_kernel", "tt_dots_kernel", "tt_norm2_dd_kernel", "gmres_team_kernel"} <= coop
    for s in srcs.values():
        for k in coop:
            assert not re.search(r"launch_pdl\(\s*" + k + r"\b", s)
