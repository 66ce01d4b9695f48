"""bench.py's multi-process path on the CPU: world size 2 over gloo (127.0.0.1).

Every rank runs its own replica; the process group carries the barriers and the
max-over-ranks timing, and the whole-job rate counts the cells of all ranks.  The
reference arm runs on rank 0 only; other ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
dist, rank, ws = bench.dist_setup("gloo")
assert (rank, ws) == (int(os.environ["RANK"]), 2)
ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)          # rank 1 is the slow one
rate = bench.whole_job_rate(ws, 1000, 3 * 4, ms)
dist.barrier()
print(json.dumps({{"rank": rank, "ms": ms, "rate": rate}}))
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(code, n=2):
    port = _port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    import json
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run(CHILD.format(root=ROOT))]
    for o in outs:
        assert o["ms"] == 15.0                               # the slowest rank
        assert o["rate"] == pytest.approx(2 * 1000 * 12 / 0.015)


def test_reference_arm_runs_on_rank_zero_only():
    code = "import sys; sys.path.insert(0, %r); import bench; bench.run_reference(bench.parse_args(['--impl', 'reference']))" % ROOT
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_port()))
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""                            # rank 1: no work, no line


def test_density_image_is_a_valid_png(tmp_path):
    """bench.py --dmr writes greyscale PNGs with its own encoder: signature, IHDR and a zlib stream
    that inflates back to the filtered rows."""
    import struct
    import zlib
    import numpy as np
    import bench
    img = (np.arange(6 * 5) * 7 % 256).astype(np.uint8).reshape(5, 6)
    path = tmp_path / "x.png"
    bench._write_png(str(path), img)
    b = path.read_bytes()
    assert b[:8] == b"\x89PNG\r\n\x1a\n"
    n, tag = struct.unpack(">I4s", b[8:16])
    assert tag == b"IHDR" and struct.unpack(">IIBBBBB", b[16:16 + n]) == (6, 5, 8, 0, 0, 0, 0)
    i = b.index(b"IDAT")
    m = struct.unpack(">I", b[i - 4:i])[0]
    raw = zlib.decompress(b[i + 4:i + 4 + m])
    rows = np.frombuffer(raw, np.uint8).reshape(5, 7)
    assert (rows[:, 0] == 0).all() and np.array_equal(rows[:, 1:], img)
    assert zlib.crc32(b[i:i + 4 + m]) & 0xFFFFFFFF == struct.unpack(">I", b[i + 4 + m:i + 8 + m])[0]
