"""B300-native adaptive-multigrid Wilson-Dirac solver (arXiv:0912.2186): libwmg.so + binding."""
from . import wmg  # noqa: F401
from .wmg import Context, Params, Info, WmgError, default_params, PREC_DOUBLE, PREC_SINGLE, PREC_HALF  # noqa: F401
