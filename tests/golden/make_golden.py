"""Writes tests/golden/config1_answer.json: the oracle's answer on the small
ER workload (1,000 vertices, 5,000 edges, 3 labels, query 0/1* from vertex 0).
Calls only the oracle and the input generators."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from oracle.regex_nfa import compile_regex  # noqa: E402
from paper_2412_10287_gb300 import workloads as W  # noqa: E402


def main():
    w = W.config1()
    g = w.graph
    q = w.queries[0]
    r = O.ssr(g.n, g.n_labels, g.src, g.dst, g.lab, compile_regex(q.regex, g.n_labels), q.source)
    out = {"workload": w.notes, "regex": q.regex, "source": q.source,
           "answer": r["answer"].tolist(), "counters": r["counters"]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_answer.json"),
              "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
