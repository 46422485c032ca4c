"""The paper's popcount forms of 1-bit dot products (Sec. III-D, III-E).

TEST INFRASTRUCTURE ONLY.  These restate, on Python integers used as bit
vectors (bit k = element k), the closed forms the paper derives; the tests
pin the int64 oracle ``oracle.bgemm`` against them and against explicit +-1
arithmetic.  Encoding (Fig. 1): bit 1 is +1, bit 0 is -1.
"""
from __future__ import annotations


def popc(v: int) -> int:
    return bin(v).count("1")


def mask(K: int) -> int:
    return (1 << K) - 1


def dot_xor(a: int, b: int, K: int) -> int:
    """Eq. 4: real 1-bit dot product K - 2 popc(A xor B)."""
    return K - 2 * popc((a ^ b) & mask(K))


def dot_and(a: int, b: int, K: int) -> int:
    """Eq. 6: 2 (popc(A and B) + popc(not A and not B)) - K."""
    m = mask(K)
    return 2 * (popc(a & b & m) + popc(~a & ~b & m)) - K


def complex_dot_padded(ar: int, ai: int, br: int, bi: int, K: int, K_pad: int):
    """Eq. 5: complex 1-bit dot product of length-K vectors that were padded
    with K_pad zero bits (value -1) to length Kp = K + K_pad.  The K in the
    paper's formula is read as the padded length Kp (the pad products cancel
    in the real part and add 2*K_pad to the imaginary part)."""
    Kp = K + K_pad
    m = mask(Kp)
    ar, ai, br, bi = ar & mask(K), ai & mask(K), br & mask(K), bi & mask(K)  # pads = 0 bits
    re = 2 * (Kp - (popc((ar ^ br) & m) + popc((ai ^ (~bi & m)) & m)))
    im = 2 * (Kp - K_pad - (popc((ar ^ bi) & m) + popc((ai ^ br) & m)))
    return re, im


def values(v: int, K: int):
    """Unpack a bit vector to +-1 integers (Fig. 1)."""
    return [1 if (v >> k) & 1 else -1 for k in range(K)]
