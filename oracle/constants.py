"""Physical constants in cgs (CODATA 2018 exact SI values, converted)."""
H_PLANCK = 6.62607015e-27      # erg s
C_LIGHT = 2.99792458e10        # cm s^-1
K_BOLTZ = 1.380649e-16         # erg K^-1
AMU = 1.66053906660e-24        # g
C2 = H_PLANCK * C_LIGHT / K_BOLTZ   # second radiation constant, cm K (1.438776877...)
T_REF = 296.0                  # HITRAN reference temperature, K
BAR = 1e6                      # dyn cm^-2 per bar
