"""Safety properties of the CUDA sources and the profiling records, checked as text (CPU only).

- Every device-side wait is bounded: the only mbarrier wait instruction sits in the one
  try-wait helper, and that helper is called only by the bounded waits built on
  %globaltimer (which return false once their budget has passed).  The grid-resident CG
  loop's waits on other blocks (an epoch counter, per-block flags) go through one helper
  that gives up after the solve's wait bound or once another block has given up.
- No device code traps or asserts: a failure is a status the host reads.
- Every ncu command recorded under profiles/ leaves the GPU clocks alone and runs only
  committed files; every capture beyond the one-pass launch list names one kernel and at most
  three launches.
"""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_1410_4054_gb300" / "csrc"


def sources():
    return sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")))


def strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_every_mbarrier_wait_is_bounded():
    sites = {p.name: strip_comments(p.read_text()).count("mbarrier.try_wait") for p in sources()}
    assert {k: v for k, v in sites.items() if v} == {"pk_tile.cuh": 1}
    tile = strip_comments((CSRC / "pk_tile.cuh").read_text())
    # the helper's callers: only the bounded waits
    heads = [(m.start(), m.group(1)) for m in
             re.finditer(r"__device__\s+__forceinline__\s+[\w:<>*&\s]+?\b(\w+)\s*\(", tile)]
    callers = set()
    for m in re.finditer(r"\bmbar_try_wait\(", tile):
        enclosing = [name for pos, name in heads if pos < m.start()]
        callers.add(enclosing[-1])
    assert callers == {"mbar_try_wait", "mbar_wait_for", "mbar_wait_st"}
    assert "global_ns() - t0 > budget_ns" in tile
    for p in sources():
        if p.name != "pk_tile.cuh":
            assert "mbar_try_wait(" not in strip_comments(p.read_text()), p.name


def test_grid_resident_waits_are_bounded():
    src = strip_comments((CSRC / "pk_resident.cu").read_text())

    def body(name):
        t = src[src.index(name):]
        return t[:t.index("\n}\n")]

    # the spins on other blocks' progress: relaxed polls, only inside the warp-wide helper,
    # which gives up after the solve's wait bound or once another block has given up
    flags = body("bool warp_wait_flags(")
    assert src.count("ld_relaxed(") == 1 + flags.count("ld_relaxed(")
    assert "global_ns() - t0 > st->wait_ns" in flags and "report_timeout(st)" in flags
    assert "__ldcg(&st->timeout)" in flags
    # the producer lane's spin on its own block's decision is bounded the same way
    dec = body("bool wait_block_decision(")
    assert "global_ns() - t0 > st->wait_ns" in dec and "report_timeout(st)" in dec
    # no other loop in the file polls memory
    assert src.count("__nanosleep(") == 2
    # all blocks resident at once: the launch is cooperative
    assert "cudaLaunchAttributeCooperative" in src


def test_no_device_traps_or_asserts():
    for p in sources():
        t = strip_comments(p.read_text())
        assert "__trap" not in t and "trap;" not in t, p.name
        assert not re.search(r"(?<!static_)\bassert\s*\(", t), p.name


def test_profiles_record_safe_ncu_commands():
    committed = {p.name for p in ROOT.iterdir()}
    for p in sorted((ROOT / "profiles").glob("*.md")):
        for line in p.read_text().splitlines():
            if not line.lstrip().startswith("ncu "):
                continue
            assert "--clock-control none" in line, (p.name, line)
            prog = re.search(r"\bpython\s+(\S+)", line)
            assert prog and prog.group(1) in committed, (p.name, line)
            # anything beyond the one-pass launch list profiles one kernel, a few launches
            if "--metrics gpu__time_duration.sum " not in line:
                k = re.search(r"-k\s+(\S+)", line)
                assert k and not re.search(r"[|\[\]()]", k.group(1)), (p.name, line)
                c = re.search(r"-c\s+(\d+)", line)
                assert c and int(c.group(1)) <= 3, (p.name, line)
