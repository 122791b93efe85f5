"""Physical constants of the oracle (SI).

gamma0 is the gyromagnetic ratio in rad/(s T).  The paper states that its
conventions follow mumax3 but prints no value; 1.7595e11 (mumax3's) is the
reading taken.  mu0 is 4 pi 1e-7 (the value mumax3 uses).
"""
import math

MU0 = 4e-7 * math.pi            # T m / A
GAMMA0 = 1.7595e11              # rad / (s T)
KB = 1.380649e-23               # J / K
HBAR = 1.054571817e-34          # J s
QE = 1.602176634e-19            # C
MU_B = 9.2740100783e-24         # J / T
