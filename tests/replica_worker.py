"""One CPU rank of the replica tests (spawned; gloo on 127.0.0.1)."""
import os


def run(rank, world, port, q):
    import torch.distributed as dist

    from paper_1403_0555_b300.replicas import rank_seed, reduce_timing
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, count = reduce_timing(dist, 10.0 + rank, 100.0 * (rank + 1))
        seeds = [rank_seed(rank, j) for j in range(8)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        dist.barrier()
        q.put((rank, ms, count, gathered))
    finally:
        dist.destroy_process_group()
