"""GB300-native (sm_103a) mechanical-interaction iteration of an agent-based
tissue simulation (BioDynaMo, PPoPP'23): uniform-grid neighbour search in
Morton order, 27-box overlap force, clamped displacement, static-agent skip and
the parallel merge of daughters created by division."""
