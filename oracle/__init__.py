"""CPU oracle (test infrastructure only): see ea_oracle.py."""
from .ea_oracle import *  # noqa: F401,F403
from .ea_oracle import lib  # noqa: F401
