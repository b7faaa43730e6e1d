"""A rank of the launcher test (not a test module): joins a gloo group with the
variables torchrun sets, checks the bookkeeping the benchmark uses, writes one JSON file."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

from paper_1301_1714_gb300 import replicas  # noqa: E402

world, rank, local_rank = replicas.rank_env()
dist.init_process_group("gloo")
n_total = replicas.reduce_sum(1000.0 * (rank + 1))
t_max = replicas.reduce_max(0.5 + rank)
with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as f:
    json.dump({"world": world, "rank": rank, "local_rank": local_rank, "group_size": dist.get_world_size(),
               "n_total": n_total, "t_max": t_max}, f)
dist.destroy_process_group()
