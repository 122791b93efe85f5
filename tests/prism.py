"""Closed-form demagnetising factors of a uniformly magnetised rectangular
prism, shared by the oracle pins (no oracle code)."""
import math


def prism_factor(a, b, c):
    """Demagnetising factor along the edge 2c of a uniformly magnetised
    rectangular prism 2a x 2b x 2c, in the closed form of A. Aharoni,
    J. Appl. Phys. 83, 3432 (1998) (derived from the prism's magnetostatic
    energy, independently of Newell's f and g functions)."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    ln = math.log
    s = ((b * b - c * c) / (2 * b * c) * ln((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * ln((r - b) / (r + b))
         + b / (2 * c) * ln((ab + a) / (ab - a)) + a / (2 * c) * ln((ab + b) / (ab - b))
         + c / (2 * a) * ln((bc - b) / (bc + b)) + c / (2 * b) * ln((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / math.pi
