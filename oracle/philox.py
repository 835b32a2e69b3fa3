"""Philox4x32-10 counter-based generator and the uniform draw used for every
random event of a shot.

Test infrastructure only: the CUDA path never imports this module.

Philox4x32-10 is defined in J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4
(the Philox S-box: two 32x32->64 multiplies per round, Weyl-sequence key
schedule, ten rounds).  The paper simulated here does not fix a random
number generator; the reading used by this project (counter layout and the
53-bit uniform) is:

    key     = (seed & 0xffffffff, seed >> 32)
    counter = (shot & 0xffffffff, shot >> 32, event_id, 0)
    u       = ((w0 << 21) ^ (w1 >> 11)) * 2**-53        in [0, 1)
"""

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9  # golden ratio
PHILOX_W1 = 0xBB67AE85  # sqrt(3) - 1


def philox4x32_10(counter, key):
    """Ten Philox rounds on a 4x32-bit counter with a 2x32-bit key."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in counter)
    k0, k1 = (int(v) & MASK32 for v in key)
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
        k0 = (k0 + PHILOX_W0) & MASK32
        k1 = (k1 + PHILOX_W1) & MASK32
    return c0, c1, c2, c3


def uniform(seed, shot, event_id):
    """The uniform in [0, 1) that event `event_id` of shot `shot` consumes."""
    w = philox4x32_10(
        (shot & MASK32, (shot >> 32) & MASK32, event_id & MASK32, 0),
        (seed & MASK32, (seed >> 32) & MASK32),
    )
    bits53 = (w[0] << 21) ^ (w[1] >> 11)
    return bits53 * (2.0 ** -53)
