"""The parse stage's codec (host only): bit-exact round trips, the byte
format against a Python statement of it (XOR with the previous value's bits,
unsigned LEB128), and rejection of malformed input."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def b():
    from paper_2009_04755_gb300 import _build
    _build.build()
    import paper_2009_04755_gb300.binding as b
    return b


def _encode_py(x):
    out = bytearray()
    prev = 0
    for u in np.ascontiguousarray(x, np.float32).view(np.uint32).tolist():
        v = u ^ prev
        prev = u
        while True:
            byte = v & 0x7F
            v >>= 7
            out.append(byte | (0x80 if v else 0))
            if not v:
                break
    return bytes(out)


def test_round_trip_and_format(b):
    rng = np.random.default_rng(0)
    for x in (rng.standard_normal(4097).astype(np.float32),
              (rng.standard_normal(300) * 1e30).astype(np.float32),
              np.zeros(17, np.float32), np.arange(1000, dtype=np.float32)):
        e = b.encode_vector(x)
        assert e == _encode_py(x)
        y = b.decode_vector(e, len(x))
        np.testing.assert_array_equal(y.view(np.uint32), x.view(np.uint32))


def test_special_values_bit_exact(b):
    bits = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00001,
                     0xFFFFFFFF, 0x00000001, 0x807FFFFF, 0x7F7FFFFF, 0x3F800000],
                    np.uint32)
    x = bits.view(np.float32)
    y = b.decode_vector(b.encode_vector(x), len(x))
    np.testing.assert_array_equal(y.view(np.uint32), bits)
    assert b.decode_vector(b.encode_vector(np.zeros(0, np.float32)), 0).size == 0


def test_malformed_input_rejected(b):
    x = np.random.default_rng(1).standard_normal(64).astype(np.float32)
    e = b.encode_vector(x)
    for bad in (e[:-1], e + b"\x00", b"\xff" * 10, e[:5]):
        with pytest.raises(b.APError):
            b.decode_vector(bad, 64)
