"""The autotuner cache's key and file round trip (host logic, no device)."""
from paper_2109_13030_b300 import tune_cache as C


def test_key_ignores_order_and_buckets_the_batch():
    a = C.key([(100, 3, 10, 1000), (50, 2, 4, 130)], 0, 148, 30)
    b = C.key([(50, 2, 4, 200), (100, 3, 10, 1024)], 0, 148, 30)
    assert a == b
    assert C.key([(100, 3, 10, 1000)], 0, 148, 30) != C.key([(100, 3, 10, 1025)], 0, 148, 30)
    assert C.key([(100, 3, 10, 1000)], 0, 148, 30) != C.key([(100, 3, 10, 1000)], 1, 148, 30)
    assert C.key([(100, 3, 10, 1000)], 0, 148, 30) != C.key([(100, 3, 10, 1000)], 0, 132, 30)
    assert C.batch_bucket(1) == 1 and C.batch_bucket(129) == 256 and C.batch_bucket(2048) == 2048
    # the problems' kernel choices are part of the key, in the shapes' order
    assert C.key([(100, 3, 10, 1000)], 0, 148, 30) == C.key([(100, 3, 10, 1000)], 0, 148, 30, [0])
    assert C.key([(100, 3, 10, 1000)], 0, 148, 30, [4]) != C.key([(100, 3, 10, 1000)], 0, 148, 30, [0])
    assert (C.key([(100, 3, 10, 1000), (50, 2, 4, 130)], 0, 148, 30, [4, 0])
            == C.key([(50, 2, 4, 130), (100, 3, 10, 1000)], 0, 148, 30, [0, 4]))


def test_store_and_lookup(tmp_path):
    path = str(tmp_path / "tune.json")
    k = C.key([(150, 4, 32, 2048)], 0, 148, 100)
    assert C.lookup(path, k) is None
    C.store(path, k, 704, 12.5)
    assert C.lookup(path, k) == (704, 12.5, 0)
    k2 = C.key([(50, 2, 2, 128)], 0, 148, 100, [4])
    C.store(path, k2, 512, 3.0, 6)
    assert C.lookup(path, k) == (704, 12.5, 0) and C.lookup(path, k2) == (512, 3.0, 6)
    # an entry written before the slot cap existed reads as "as many as fit"
    import json
    data = json.load(open(path))
    data[k] = {"threads": 384, "ms": 1.0}
    json.dump(data, open(path, "w"))
    assert C.lookup(path, k) == (384, 1.0, 0)
    open(path, "w").write("not json")
    assert C.lookup(path, k) is None
