"""Method coefficient tables of the oracle (binary64).

TEST INFRASTRUCTURE ONLY.  Written by oracle/derive_coefficients.py; the
derivation and the order conditions are stated in that file.
"""

# ROK4: Eq. ROK with s = 4; alpha and b are the classical RK4 tableau.
ROK4_GAMMA = 0.5728160624821349
ROK4_ALPHA = [[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]
ROK4_GAMMA_OFFDIAG = [[0.0, 0.0, 0.0, 0.0], [0.025068629909359066, 0.0, 0.0, 0.0], [0.2477474325727758, -1.405913872491725, 0.0, 0.0], [0.6, -0.020369905583413464, -1.7503308492902152, 0.0]]
ROK4_B = [0.16666666666666666, 0.3333333333333333, 0.3333333333333333, 0.16666666666666666]

# classical RK4 (Sec. 2.1, Eq. RK with a, b below)
RK4_A = [[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]
RK4_B = [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]

# ESDIRK3: explicit first stage, diagonal gamma, stiffly accurate (b = last row)
# R(inf) = 0 numerator polynomial in gamma: 6*x**3 - 18*x**2 + 9*x - 1
ESDIRK3_GAMMA = 0.435866521508459
ESDIRK3_A = [[0.0, 0.0, 0.0, 0.0], [0.435866521508459, 0.435866521508459, 0.0, 0.0], [0.2576482460664272, -0.09351476757488625, 0.435866521508459, 0.0], [0.18764102434672383, -0.595297473576955, 0.9717899277217721, 0.435866521508459]]
ESDIRK3_B = [0.18764102434672383, -0.595297473576955, 0.9717899277217721, 0.435866521508459]
ESDIRK3_C = [0.0, 0.871733043016918, 0.6, 1.0]
