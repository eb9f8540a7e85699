"""The committed warm-start networks are well-formed blobs of the layout
zema_load_warmstart reads (magic, layer count, widths, then FP32 weights and
biases layer by layer), with the widths their metadata records: the
per-vertex network 13 -> 128^3 -> 3 and the per-body network 40 -> 128^3 ->
12.  The held-out evaluation record is internally consistent."""
import json
import os

import numpy as np

from paper_2311_05945_b300 import zema as Z

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2311_05945_b300",
                       "weights")


def _n_params(dims):
    return sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))


def test_warmstart_blobs_match_their_metadata():
    for name, dims_expect in (("warmstart", [13, 128, 128, 128, 3]), ("warmstart_affine", [40, 128, 128, 128, 12])):
        blob = open(os.path.join(WEIGHTS, name + ".bin"), "rb").read()
        meta = json.load(open(os.path.join(WEIGHTS, name + ".json")))
        head = np.frombuffer(blob[:8], dtype=np.uint32)
        assert head[0] == 0x5357455A and head[1] == len(dims_expect) - 1
        dims, theta = Z.read_warmstart_blob(blob)
        assert dims == dims_expect == meta["dims"]
        assert len(blob) == 4 * (2 + len(dims)) + 4 * _n_params(dims)
        assert theta.size == _n_params(dims) and np.all(np.isfinite(theta))
        # trained: the biases have moved from their zero initialisation
        off = 0
        for a, b in zip(dims[:-1], dims[1:]):
            off += a * b
            assert np.any(theta[off:off + b] != 0.0)
            off += b
        assert bytes(Z.warmstart_blob(dims, theta)) == blob


def test_evaluation_record_is_consistent():
    ev = json.load(open(os.path.join(WEIGHTS, "warmstart_eval.json")))
    cv, lr = ev["constant_velocity"], ev["learned"]
    assert ev["envs"] == 64 and ev["seed0"] == 100000
    assert abs(ev["newton_ratio"] - lr["newton_iters"] / cv["newton_iters"]) < 1e-12
    for r in (cv, lr):
        # batch steps (all 64 envs at once) per second
        assert abs(r["steps_per_s"] - ev["steps"] / r["seconds"]) < 1e-9 * r["steps_per_s"]
    assert cv["warm_learned"] == 0 and lr["warm_learned"] > 0
