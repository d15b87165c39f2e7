"""B300-native field-window estimator (xi, xi_l, zeta_l) behind the libhermes C ABI."""
from .hermes import (Context, HermesError, Server, estimate_bytes, fft_set_variant, fft_variants,  # noqa: F401
                     shell_table_host)
