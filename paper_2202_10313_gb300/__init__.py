"""GB300-native ADER-DG + clustered local time stepping (package root)."""
