"""CPU oracle of PDLP — test infrastructure only (see ``pdlp_oracle``)."""
from .pdlp_oracle import *  # noqa: F401,F403
from . import pdlp_oracle  # noqa: F401
