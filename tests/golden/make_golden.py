"""Write tests/golden/workloads.json: expected counts of the large seeded
workloads, computed by the CPU oracle only (O2 for the large graphs, O1 for the
small one, both cross-checked where affordable).

For every workload it stores the SHA-256 of the generated CSR (so a test can
tell that the generator produced the same graph on another machine), the 15
global counts, and the SHA-256 of the per-edge count matrix (uint64 [m, 15],
little-endian, CSR edge order) where per-edge counts are part of the workload.

    python tests/golden/make_golden.py [erdos_renyi_small chung_lu_1m rmat_22]
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_1506_04322_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")


def csr_sha(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype="<i4").tobytes())
    return h.hexdigest()


def matrix_sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        t0 = time.time()
        g = getattr(inputs, name)()
        rec = {"n": g.n, "m": g.m, "csr_sha256": csr_sha(g), "max_degree": int(g.degrees().max())}
        if name == "erdos_renyi_small":
            glob = oracle.alg2_global(g)
            pe = oracle.alg2_per_edge(g)
            assert glob == oracle.o2_global(g)
            assert np.array_equal(pe, oracle.o2_per_edge(g))
            rec["global"] = [str(x) for x in glob]
            rec["per_edge_sha256"] = matrix_sha(pe)
            rec["method"] = "O1 literal Algorithm 2 (checked against O2)"
        elif name == "chung_lu_1m":
            pe = oracle.o2_per_edge(g, threads=0)
            glob = oracle.o2_global(g, threads=0)
            rec["global"] = [str(x) for x in glob]
            rec["per_edge_sha256"] = matrix_sha(pe)
            rec["method"] = "O2 independent method"
        else:
            glob = oracle.o2_global(g, threads=0)
            rec["global"] = [str(x) for x in glob]
            rec["method"] = "O2 independent method"
        rec["oracle_seconds"] = round(time.time() - t0, 1)
        data[name] = rec
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(name, rec["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["erdos_renyi_small", "chung_lu_1m", "rmat_22"])
