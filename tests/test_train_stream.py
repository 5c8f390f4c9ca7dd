"""The trainer's streamed systems are the batch-generated ones, in order
(CPU; the spawn pool holds no CUDA context)."""
import numpy as np


def test_streamed_systems_equal_batch_systems():
    from paper_1912_04385_gb300 import train_gnn as T
    batch, pes = T.make_systems(5, 12, seed=3, workers=2)
    streamed = list(T.stream_systems(5, 12, seed=3, workers=2, chunk=2))
    assert len(streamed) == len(batch) == 5
    for a, b in zip(streamed, batch):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert len(set(pes)) == 5 and all(0.1 <= p <= 1000.0 for p in pes)
