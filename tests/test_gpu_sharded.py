"""The sharded Alg. 3 driver on the GPU backend (one rank, NCCL): the merge
scoring goes through csvd_score and the state exchange through NCCL
broadcasts; the clusters equal the FP64 oracle's (the multi-rank logic
itself is checked with two gloo ranks on the CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist

from oracle import cluster as ocluster
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("chunk", [4, 64])
def test_sharded_driver_on_gpu_matches_oracle(cuda_lib, chunk):
    from paper_2601_11626_gb300 import sharded
    col = synth.small_c1()
    r, eps = col.meta["r"], col.meta["eps"]
    want = ocluster.cluster(col.blocks, r, eps, "approx", "frobenius")
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        be = sharded.CsvdBackend([b.cuda() for b in col.blocks], r, eps, "mixed")
        labels, clusters, est = sharded.cluster_approx_sharded(be, len(col.blocks), eps,
                                                               chunk=chunk, device="cuda")
    finally:
        dist.destroy_process_group()
    assert labels == want["labels"]
    assert clusters == want["clusters"]
    for a, b, e in zip(est, want["estimate_sq"], want["energy"]):
        assert abs(a - b) <= 2e-4 * b + 4 * 2.0 ** -24 * e
