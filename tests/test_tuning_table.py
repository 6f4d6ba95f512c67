"""The launch-shape table of the autotuner: defaults, validation, install and
reset (host logic only; no GPU call)."""
import pytest

from paper_2508_11443_b300 import build as B


@pytest.fixture(scope="module")
def F():
    B.build()
    from paper_2508_11443_b300 import fks
    yield fks
    fks.fks_tuning_reset()


def test_defaults(F):
    F.fks_tuning_reset()
    t = F.fks_tuning_get(F.FKS_KEY_U64, 1)
    assert (t.thread_search_max, t.part_ctas_per_sm, t.scatter_blocks_per_sm, t.split_min_keys_log2) == (3, 0, 8, 20)
    assert (t.lookup_queries_per_thread, t.lookup_block, t.lookup_blocks_per_sm) == (4, 256, 8)
    assert t.tuned == 0 and t.part_prefetch == 1
    # with 8 or 16 keys per bucket every bucket of two or more keys goes to a
    # warp segment; with 16, partitions take their next ticket only when free
    t16 = F.fks_tuning_get(F.FKS_KEY_BYTES, 16)
    assert t16.thread_search_max == 1 and t16.part_prefetch == 0
    assert F.fks_tuning_get(F.FKS_KEY_U64, 8).part_prefetch == 1


def test_install_and_reset(F):
    F.fks_tuning_reset()
    t = F.fks_tuning_get(F.FKS_KEY_U64, 4)
    t.thread_search_max, t.lookup_block, t.lookup_queries_per_thread = 2, 512, 8
    F.fks_tuning_set(t)
    got = F.fks_tuning_get(F.FKS_KEY_U64, 4)
    assert (got.thread_search_max, got.lookup_block, got.lookup_queries_per_thread) == (2, 512, 8)
    # other (kind, lambda) entries keep their defaults
    assert F.fks_tuning_get(F.FKS_KEY_U64, 1).thread_search_max == 3
    assert F.fks_tuning_get(F.FKS_KEY_BYTES, 4).lookup_block == 256
    F.fks_tuning_reset()
    assert F.fks_tuning_get(F.FKS_KEY_U64, 4).thread_search_max == 3


@pytest.mark.parametrize("field,value", [("thread_search_max", 0), ("thread_search_max", 4),
                                         ("part_ctas_per_sm", 3), ("scatter_blocks_per_sm", 0),
                                         ("split_min_keys_log2", 9), ("lookup_queries_per_thread", 3),
                                         ("lookup_block", 1024), ("lookup_blocks_per_sm", 0),
                                         ("lookup_blocks_per_sm", 1025),
                                         ("keys_per_bucket", 3), ("key_kind", 2), ("part_prefetch", 2)])
def test_out_of_range_entries_are_rejected(F, field, value):
    t = F.fks_tuning_get(F.FKS_KEY_U64, 1)
    setattr(t, field, value)
    with pytest.raises(F.FksError) as e:
        F.fks_tuning_set(t)
    assert e.value.status == F.FKS_ERR_INVALID_ARG


def test_bad_keys_per_bucket_is_rejected(F):
    with pytest.raises(F.FksError):
        F.fks_tuning_get(F.FKS_KEY_U64, 3)


def test_save_and_load_round_trip(F, tmp_path):
    F.fks_tuning_reset()
    a = F.fks_tuning_get(F.FKS_KEY_U64, 1)
    a.lookup_block, a.lookup_blocks_per_sm, a.tuned, a.build_ms, a.sample_keys = 512, 1024, 1, 3.98, 1 << 26
    F.fks_tuning_set(a)
    b = F.fks_tuning_get(F.FKS_KEY_BYTES, 16)
    b.thread_search_max, b.split_min_keys_log2, b.part_prefetch = 2, 22, 1
    F.fks_tuning_set(b)
    path = str(tmp_path / "tune.txt")
    F.fks_tuning_save(path)
    F.fks_tuning_reset()
    assert F.fks_tuning_get(F.FKS_KEY_U64, 1).lookup_block == 256
    F.fks_tuning_load(path)
    got_a, got_b = F.fks_tuning_get(F.FKS_KEY_U64, 1), F.fks_tuning_get(F.FKS_KEY_BYTES, 16)
    assert (got_a.lookup_block, got_a.lookup_blocks_per_sm, got_a.tuned, got_a.sample_keys) == (512, 1024, 1, 1 << 26)
    assert abs(got_a.build_ms - 3.98) < 1e-4
    assert (got_b.thread_search_max, got_b.split_min_keys_log2, got_b.part_prefetch) == (2, 22, 1)
    F.fks_tuning_reset()
    # a line of the first format (no part_prefetch) takes the default for its lambda
    (tmp_path / "v1.txt").write_text("fks_tuning 1 0 16 2 0 8 20 4 512 8 1 1.0 1.0 100\n"
                                     "fks_tuning 1 0 8 2 0 8 20 4 512 8 1 1.0 1.0 100\n")
    F.fks_tuning_load(str(tmp_path / "v1.txt"))
    v16, v8 = F.fks_tuning_get(F.FKS_KEY_U64, 16), F.fks_tuning_get(F.FKS_KEY_U64, 8)
    assert (v16.thread_search_max, v16.lookup_block, v16.part_prefetch) == (2, 512, 0)
    assert v8.part_prefetch == 1
    F.fks_tuning_reset()


def test_malformed_tuning_file_installs_nothing(F, tmp_path):
    F.fks_tuning_reset()
    path = tmp_path / "bad.txt"
    path.write_text("fks_tuning 1 0 1 2 0 8 20 4 512 8 1 1.0 1.0 100\n"
                    "fks_tuning 1 0 4 9 0 8 20 4 256 8 1 1.0 1.0 100\n")  # thread_search_max 9: out of range
    with pytest.raises(F.FksError):
        F.fks_tuning_load(str(path))
    assert F.fks_tuning_get(F.FKS_KEY_U64, 1).thread_search_max == 3  # the good first line was not installed
    with pytest.raises(F.FksError):
        F.fks_tuning_load(str(tmp_path / "missing.txt"))
