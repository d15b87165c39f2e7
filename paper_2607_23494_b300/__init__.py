"""B300-native field-window estimator (xi, xi_l, zeta_l) behind the libhermes C ABI."""
from .hermes import Context, HermesError, Server, estimate_bytes, shell_table_host  # noqa: F401
