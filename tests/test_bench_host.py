"""Host logic of bench.py that needs no GPU: the source hash that ties the
stored ncu counters of a kernel to the text of that kernel."""
import hashlib

import bench


def _h(*parts: bytes) -> str:
    h = hashlib.sha256()
    for p in parts:
        h.update(p)
    return h.hexdigest()[:16]


def test_sources_hash_ranges(tmp_path):
    (tmp_path / "a.cu").write_bytes(b"helpers\n// cut one\nbound pass\n// start two\nkernel\n// end two\nhost\n")
    (tmp_path / "b.cuh").write_bytes(b"header\n")
    whole = bench.sources_hash(["a.cu", "b.cuh"], root=str(tmp_path))
    assert whole == _h(b"helpers\n// cut one\nbound pass\n// start two\nkernel\n// end two\nhost\n", b"header\n")
    ranged = bench.sources_hash([("a.cu", None, "// cut one"), ("a.cu", "// start two", "// end two"), "b.cuh"],
                                root=str(tmp_path))
    assert ranged == _h(b"helpers\n", b"// start two\nkernel\n", b"header\n")
    # text outside the ranges does not move the hash; text inside does
    (tmp_path / "a.cu").write_bytes(b"helpers\n// cut one\nBOUND PASS\n// start two\nkernel\n// end two\nHOST\n")
    assert bench.sources_hash([("a.cu", None, "// cut one"), ("a.cu", "// start two", "// end two"), "b.cuh"],
                              root=str(tmp_path)) == ranged
    (tmp_path / "a.cu").write_bytes(b"helpers\n// cut one\nbound pass\n// start two\nkernel2\n// end two\nhost\n")
    assert bench.sources_hash([("a.cu", None, "// cut one"), ("a.cu", "// start two", "// end two"), "b.cuh"],
                              root=str(tmp_path)) != ranged
    # a missing start marker hashes nothing of that file (the stored counters then do not apply)
    assert bench.sources_hash([("a.cu", "// absent", None)], root=str(tmp_path)) == _h(b"")


def test_element_kernel_ranges_exist():
    """The markers that delimit the element kernel's text are present once in
    the source, so the hash covers the kernel and not an empty range."""
    for path, start, end in [e for e in bench.MIXED_ELEM_NCU["sources"] if not isinstance(e, str)]:
        text = open(bench.os.path.join(bench.ROOT, path), encoding="utf-8").read()
        for m in (start, end):
            if m is not None:
                assert text.count(m) == 1, m
        if start is not None and end is not None:
            assert text.index(start) < text.index(end)
