"""The batch autotuner's cache file, through the host-only boundary calls
(no device needed): lookup of missing files and keys, the last entry of a
key winning, malformed and out-of-range lines ignored, argument checks."""
import pytest

import paper_2512_11473_b300 as sg


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_11473_b300 import build
    build.build()


def test_missing_file_is_an_empty_cache(tmp_path):
    assert sg.autotune_cache_lookup(tmp_path / "none.txt", "k") is None


def test_store_then_lookup_last_entry_wins(tmp_path):
    p = tmp_path / "c.txt"
    sg.autotune_cache_store(p, "gpu=X;sweeps=20", 4, 1)
    sg.autotune_cache_store(p, "gpu=Y;sweeps=20", 2, 2)
    assert sg.autotune_cache_lookup(p, "gpu=X;sweeps=20") == (4, 1)
    assert sg.autotune_cache_lookup(p, "gpu=Y;sweeps=20") == (2, 2)
    sg.autotune_cache_store(p, "gpu=X;sweeps=20", 8, 2)
    assert sg.autotune_cache_lookup(p, "gpu=X;sweeps=20") == (8, 2)
    assert sg.autotune_cache_lookup(p, "gpu=X;sweeps=2") is None  # keys match whole
    assert p.read_text().splitlines() == ["gpu=X;sweeps=20 4 1", "gpu=Y;sweeps=20 2 2", "gpu=X;sweeps=20 8 2"]


def test_malformed_and_invalid_lines_are_ignored(tmp_path):
    p = tmp_path / "c.txt"
    p.write_text("k 4 1\nk 3 1\nk 2 2 trailing\nk x y\n\nk\nk 1 2\nk 16 1\n")
    # "k 2 2 trailing" parses as (2, 2); (3, 1), (1, 2) and (16, 1) are no candidates
    assert sg.autotune_cache_lookup(p, "k") == (2, 2)


@pytest.mark.parametrize("key,ppi,dep", [("has space", 4, 1), ("", 4, 1), ("k", 3, 1), ("k", 1, 2), ("k", 4, 3),
                                         ("x" * 400, 4, 1)])
def test_store_rejects_bad_arguments(tmp_path, key, ppi, dep):
    with pytest.raises(sg.SgError) as e:
        sg.autotune_cache_store(tmp_path / "c.txt", key, ppi, dep)
    assert e.value.status == sg.SG_ERR_INVALID
    assert not (tmp_path / "c.txt").exists()


def test_store_to_an_unwritable_path_is_an_io_error(tmp_path):
    with pytest.raises(sg.SgError) as e:
        sg.autotune_cache_store(tmp_path / "no_such_dir" / "c.txt", "k", 4, 1)
    assert e.value.status == sg.SG_ERR_IO
